// C-ABI of libvfmm: handle management, tree build and the evaluation pipeline
// P2M -> M2M -> (FP64 root + periodic lattice operator) -> M2L -> L2L -> L2P -> P2P.
// In the FP32 velocity/stretching evaluation the far-field chain (P2M ... L2P) runs on a
// handle-owned high-priority stream beside the P2P on the caller's stream, and a last kernel
// scatters the far field onto the outputs once both are done.
#include "common.cuh"
#include "vfmm_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>

struct vfmm_ctx {
    vfmm::Ctx c;
};

using namespace vfmm;

namespace {

int fail(Ctx *c, int code, const std::string &msg)
{
    if (c) c->last_error = msg;
    return code;
}

int cuda_fail(Ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? VFMM_ERR_OOM : VFMM_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

int ensure(Ctx *c, DevBuf &b, size_t bytes, const char *what)
{
    if (b.bytes >= bytes && b.p) return VFMM_OK;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return cuda_fail(c, e, what);
    }
    b.bytes = bytes;
    return VFMM_OK;
}

void release(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

template <typename T> std::vector<T> to_at(const std::vector<double> &A, int nc, int pc)
{
    // A is [nc out][nc in] row-major; AT is [pc in][OUT_ROWS out]
    std::vector<T> AT((size_t)pc * OUT_ROWS, T(0));
    for (int k = 0; k < nc; ++k)
        for (int j = 0; j < nc; ++j) AT[(size_t)j * OUT_ROWS + k] = (T)A[(size_t)k * nc + j];
    return AT;
}

// Round-to-nearest-even float -> bfloat16 bits (finite inputs).
inline uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
inline float bf16_value(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
// Round to the TF32 grid (10 explicit mantissa bits, ties away from zero), kept as float.
inline float tf32_value(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u = (u + 0x1000u) & ~0x1FFFu;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Tensor-core operand tiles: for each matrix and each TC_KBYTES-byte K chunk, the 128-row tile
// in the canonical no-swizzle K-major layout: byte (k/8)*(TC_KG*128) + kgroup*128 + (k%8)*16 +
// (byte in group).
void tile_matrix(const std::vector<double> &A, int nc, int pc, bool bf16, unsigned char *hi, unsigned char *lo)
{
    const int esz = bf16 ? 2 : 4;
    const int kc = TC_KBYTES / esz;
    const int nchunk = pc / kc;
    for (int ch = 0; ch < nchunk; ++ch) {
        unsigned char *th = hi + (size_t)ch * TC_A_TILE, *tl = lo + (size_t)ch * TC_A_TILE;
        for (int k = 0; k < 128; ++k)
            for (int e = 0; e < kc; ++e) {
                int j = ch * kc + e;
                double a = (k < nc && j < nc) ? A[(size_t)k * nc + j] : 0.0;
                size_t byte = (size_t)(k / 8) * (TC_KG * 128) + (size_t)((e * esz) / 16) * 128 +
                              (size_t)(k % 8) * 16 + (size_t)((e * esz) % 16);
                if (bf16) {
                    uint16_t h = bf16_bits((float)a);
                    uint16_t l = bf16_bits((float)(a - (double)bf16_value(h)));
                    std::memcpy(th + byte, &h, 2);
                    std::memcpy(tl + byte, &l, 2);
                } else {
                    float h = tf32_value((float)a);
                    float l = tf32_value((float)(a - (double)h));
                    std::memcpy(th + byte, &h, 4);
                    std::memcpy(tl + byte, &l, 4);
                }
            }
    }
}

inline int tindex(int tx, int ty, int tz) { return ((tx + 3) * 7 + (ty + 3)) * 7 + (tz + 3); }

template <typename T> int upload_vec(Ctx *c, DevBuf &b, const std::vector<T> &v, const char *what)
{
    int st = ensure(c, b, v.size() * sizeof(T), what);
    if (st) return st;
    cudaError_t e = cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return VFMM_OK;
}

template <typename T> int build_operators(Ctx *c)
{
    const int p = c->p, nc = c->nc, pc = c->pc;
    // M2L: k-block offset t (source = target + t) uses the operator of d = target - source = -t
    std::vector<T> m2l((size_t)NT * pc * OUT_ROWS, T(0));
    const bool tc = c->cfg.m2l_prec == VFMM_M2L_TF32X3 || c->cfg.m2l_prec == VFMM_M2L_BF16X3;
    const bool bf16 = c->cfg.m2l_prec == VFMM_M2L_BF16X3;
    const size_t tile_bytes = (size_t)pc * (bf16 ? 2 : 4) / TC_KBYTES * TC_A_TILE;  // all K chunks of one matrix
    std::vector<unsigned char> thi, tlo;
    if (tc) {
        thi.assign((size_t)NT * tile_bytes, 0);
        tlo.assign((size_t)NT * tile_bytes, 0);
    }
    for (int tx = -3; tx <= 3; ++tx)
        for (int ty = -3; ty <= 3; ++ty)
            for (int tz = -3; tz <= 3; ++tz) {
                if (std::abs(tx) <= 1 && std::abs(ty) <= 1 && std::abs(tz) <= 1) continue;
                double d[3] = {-(double)tx, -(double)ty, -(double)tz};
                std::vector<double> A = ops::m2l_hat(d, p);
                std::vector<T> at = to_at<T>(A, nc, pc);
                int ti = tindex(tx, ty, tz);
                std::copy(at.begin(), at.end(), m2l.begin() + (size_t)ti * pc * OUT_ROWS);
                if (tc) tile_matrix(A, nc, pc, bf16, thi.data() + ti * tile_bytes, tlo.data() + ti * tile_bytes);
            }
    std::vector<T> m2m((size_t)8 * pc * OUT_ROWS), l2l((size_t)8 * pc * OUT_ROWS);
    std::vector<double> m2m64((size_t)8 * nc * nc);
    for (int b = 0; b < 8; ++b) {
        int bx = (b >> 2) & 1, by = (b >> 1) & 1, bz = b & 1;
        double e1[3] = {(bx - 0.5) / 2.0, (by - 0.5) / 2.0, (bz - 0.5) / 2.0};
        std::vector<double> A = ops::m2m_hat(e1, 2.0, p);
        std::copy(A.begin(), A.end(), m2m64.begin() + (size_t)b * nc * nc);
        std::vector<T> at = to_at<T>(A, nc, pc);
        std::copy(at.begin(), at.end(), m2m.begin() + (size_t)b * pc * OUT_ROWS);
        double e2[3] = {bx - 0.5, by - 0.5, bz - 0.5};
        std::vector<T> at2 = to_at<T>(ops::l2l_hat(e2, p), nc, pc);
        std::copy(at2.begin(), at2.end(), l2l.begin() + (size_t)b * pc * OUT_ROWS);
    }
    std::vector<double> lat = ops::lattice_operator(p, c->cfg.periodic_levels);
    int st;
    if ((st = upload_vec(c, c->at_m2l, m2l, "M2L operators"))) return st;
    if (tc) {
        if ((st = upload_vec(c, c->tc_hi, thi, "tensor-core M2L tiles"))) return st;
        if ((st = upload_vec(c, c->tc_lo, tlo, "tensor-core M2L tiles"))) return st;
    }
    if ((st = upload_vec(c, c->at_m2m, m2m, "M2M operators"))) return st;
    if ((st = upload_vec(c, c->at_l2l, l2l, "L2L operators"))) return st;
    if ((st = upload_vec(c, c->m2m_f64, m2m64, "FP64 M2M operators"))) return st;
    if ((st = upload_vec(c, c->lattice_f64, lat, "lattice operator"))) return st;
    if ((st = ensure(c, c->root_m, 3 * nc * sizeof(double), "root multipole"))) return st;

    // k-block lists
    std::vector<int4> kb;
    for (int R = 1; R <= 2; ++R)
        for (int g = 0; g < 8; ++g) {
            int gx = (g >> 2) & 1, gy = (g >> 1) & 1, gz = g & 1;
            c->kb_m2l_off[R][g] = (int)kb.size();
            // children of the parent's 27 neighbours, minus the target's own (2R+1)^3 near field
            for (int Tx = -1; Tx <= 1; ++Tx)
                for (int Ty = -1; Ty <= 1; ++Ty)
                    for (int Tz = -1; Tz <= 1; ++Tz)
                        for (int b = 0; b < 8; ++b) {
                            int tx = 2 * Tx + ((b >> 2) & 1) - gx;
                            int ty = 2 * Ty + ((b >> 1) & 1) - gy;
                            int tz = 2 * Tz + (b & 1) - gz;
                            if (std::abs(tx) <= R && std::abs(ty) <= R && std::abs(tz) <= R) continue;
                            kb.push_back(make_int4(tindex(tx, ty, tz), tx, ty, tz));
                        }
            c->kb_m2l_cnt[R][g] = (int)kb.size() - c->kb_m2l_off[R][g];
        }
    c->kb_m2m_off = (int)kb.size();
    for (int b = 0; b < 8; ++b) kb.push_back(make_int4(b, (b >> 2) & 1, (b >> 1) & 1, b & 1));
    for (int g = 0; g < 8; ++g) {
        c->kb_l2l_off[g] = (int)kb.size();
        kb.push_back(make_int4(g, 0, 0, 0));
    }
    if ((st = upload_vec(c, c->kblocks, kb, "k-block lists"))) return st;
    std::vector<int4> cls;
    for (int R = 1; R <= 2; ++R)
        for (int g = 0; g < 8; ++g) {
            c->cls_off[R][g] = (int)(cls.size() / 3);
            build_line_classes(kb, c->kb_m2l_off[R][g], c->kb_m2l_cnt[R][g], g, cls);
            c->cls_cnt[R][g] = (int)(cls.size() / 3) - c->cls_off[R][g];
            if (c->cls_cnt[R][g] > 96) return fail(c, VFMM_ERR_UNSUPPORTED, "M2L offset classes exceed 96");
        }
    if ((st = upload_vec(c, c->cls, cls, "M2L offset classes"))) return st;
    return VFMM_OK;
}

// Transposed operators of the adjoint: at index t of the M2L set the transpose of the forward
// operator of offset -t (the interaction lists are symmetric, so the same lists apply), L2L_b^T
// and M2M_b^T for the child octants, and the tensor-core tiles of the transposed M2L set.
std::vector<double> transpose_sq(const std::vector<double> &A, int nc)
{
    std::vector<double> B(A.size());
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j) B[(size_t)j * nc + i] = A[(size_t)i * nc + j];
    return B;
}

template <typename T> int build_transposed(Ctx *c)
{
    const int p = c->p, nc = c->nc, pc = c->pc;
    const bool tc = c->cfg.m2l_prec == VFMM_M2L_TF32X3 || c->cfg.m2l_prec == VFMM_M2L_BF16X3;
    const bool bf16 = c->cfg.m2l_prec == VFMM_M2L_BF16X3;
    const size_t tile_bytes = (size_t)pc * (bf16 ? 2 : 4) / TC_KBYTES * TC_A_TILE;
    std::vector<T> m2l((size_t)NT * pc * OUT_ROWS, T(0));
    std::vector<unsigned char> thi, tlo;
    if (tc) {
        thi.assign((size_t)NT * tile_bytes, 0);
        tlo.assign((size_t)NT * tile_bytes, 0);
    }
    for (int tx = -3; tx <= 3; ++tx)
        for (int ty = -3; ty <= 3; ++ty)
            for (int tz = -3; tz <= 3; ++tz) {
                if (std::abs(tx) <= 1 && std::abs(ty) <= 1 && std::abs(tz) <= 1) continue;
                // the forward operator of offset -t translates by d = t
                double d[3] = {(double)tx, (double)ty, (double)tz};
                std::vector<double> A = transpose_sq(ops::m2l_hat(d, p), nc);
                std::vector<T> at = to_at<T>(A, nc, pc);
                const int ti = tindex(tx, ty, tz);
                std::copy(at.begin(), at.end(), m2l.begin() + (size_t)ti * pc * OUT_ROWS);
                if (tc) tile_matrix(A, nc, pc, bf16, thi.data() + ti * tile_bytes, tlo.data() + ti * tile_bytes);
            }
    std::vector<T> m2m((size_t)8 * pc * OUT_ROWS), l2l((size_t)8 * pc * OUT_ROWS);
    for (int b = 0; b < 8; ++b) {
        int bx = (b >> 2) & 1, by = (b >> 1) & 1, bz = b & 1;
        double e1[3] = {(bx - 0.5) / 2.0, (by - 0.5) / 2.0, (bz - 0.5) / 2.0};
        std::vector<T> a1 = to_at<T>(transpose_sq(ops::m2m_hat(e1, 2.0, p), nc), nc, pc);
        std::copy(a1.begin(), a1.end(), m2m.begin() + (size_t)b * pc * OUT_ROWS);
        double e2[3] = {bx - 0.5, by - 0.5, bz - 0.5};
        std::vector<T> a2 = to_at<T>(transpose_sq(ops::l2l_hat(e2, p), nc), nc, pc);
        std::copy(a2.begin(), a2.end(), l2l.begin() + (size_t)b * pc * OUT_ROWS);
    }
    int st;
    if ((st = upload_vec(c, c->at_m2l_t, m2l, "transposed M2L operators"))) return st;
    if ((st = upload_vec(c, c->at_m2m_t, m2m, "transposed M2M operators"))) return st;
    if ((st = upload_vec(c, c->at_l2l_t, l2l, "transposed L2L operators"))) return st;
    if (tc) {
        if ((st = upload_vec(c, c->tc_hi_t, thi, "transposed tensor-core M2L tiles"))) return st;
        if ((st = upload_vec(c, c->tc_lo_t, tlo, "transposed tensor-core M2L tiles"))) return st;
    }
    c->have_transposed = true;
    return VFMM_OK;
}

// The transposed far field of the strengths in c->gs (sorted): lambda_D = E^T w, then for each
// level from the leaves up mu_l = M2L^T lambda_l and lambda_(l-1) = L2L^T lambda_l, the root
// (mu_1 += M2M_root^T lattice^T lambda_0 when there are periodic super-levels), and from the
// root down mu_(l+1) += M2M^T mu_l.  lambda lives in the local buffer, mu in the multipole
// buffer; the leaf mu is left for launch_dual_l2p.  R: near rings of the leaf level.
int far_transpose(Ctx *c, int R)
{
    const int D = c->depth, S = c->cfg.periodic_levels;
    const int4 *kbd = (const int4 *)c->kblocks.p;
    auto lvl = [&](DevBuf &b, int l) { return (void *)((char *)b.p + c->lvl_off[l] * c->esz); };
    int rc;
    if ((rc = launch_dual_p2m(c, c->gs.p))) return rc;
    const bool tc = c->cfg.m2l_prec == VFMM_M2L_TF32X3 || c->cfg.m2l_prec == VFMM_M2L_BF16X3;
    const bool bf = c->cfg.m2l_prec == VFMM_M2L_BF16X3;
    for (int l = D; l >= 1; --l) {
        const int Rl = (l == D) ? R : 1;
        if (tc && l >= 3) {
            // the tensor-core M2L reads the multipole buffer and writes the local buffer: swap the
            // roles of the buffers and the tile sets for the transposed translation
            std::swap(c->mexp, c->lexp);
            std::swap(c->tc_hi, c->tc_hi_t);
            std::swap(c->tc_lo, c->tc_lo_t);
            rc = launch_split(c, l, bf);
            if (!rc) rc = launch_tc_m2l(c, l, Rl, bf);
            std::swap(c->mexp, c->lexp);
            std::swap(c->tc_hi, c->tc_hi_t);
            std::swap(c->tc_lo, c->tc_lo_t);
            if (rc) return rc;
        } else {
            GemmParams gp = {};
            gp.AT = c->at_m2l_t.p;
            gp.B = lvl(c->lexp, l);
            gp.C = lvl(c->mexp, l);
            gp.kb = kbd;
            for (int g = 0; g < 8; ++g) {
                gp.kb_off[g] = c->kb_m2l_off[Rl][g];
                gp.kb_cnt[g] = c->kb_m2l_cnt[Rl][g];
            }
            gp.n_src = gp.n_tgt = 1 << l;
            gp.mode = 0;
            gp.grouped = 1;
            gp.accumulate = 0;
            gp.pc = c->pc;
            if ((rc = launch_gemm(c, gp, 8, (int64_t)1 << (3 * (l - 1))))) return rc;
        }
        if (l >= 2 || S > 0) {
            // lambda_(l-1)[P] = sum_b L2L_b^T lambda_l[2P + b]
            GemmParams gp = {};
            gp.AT = c->at_l2l_t.p;
            gp.B = lvl(c->lexp, l);
            gp.C = lvl(c->lexp, l - 1);
            gp.kb = kbd;
            gp.kb_off[0] = c->kb_m2m_off;
            gp.kb_cnt[0] = 8;
            gp.n_src = 1 << l;
            gp.n_tgt = 1 << (l - 1);
            gp.mode = 1;
            gp.grouped = 0;
            gp.accumulate = 0;
            gp.pc = c->pc;
            if ((rc = launch_gemm(c, gp, 1, (int64_t)1 << (3 * (l - 1))))) return rc;
        }
    }
    if (S > 0 && (rc = launch_root_t(c))) return rc;
    for (int l = 1; l < D; ++l) {
        // mu_(l+1)[c] += M2M_(parity c)^T mu_l[c >> 1]
        GemmParams gp = {};
        gp.AT = c->at_m2m_t.p;
        gp.B = lvl(c->mexp, l);
        gp.C = lvl(c->mexp, l + 1);
        gp.kb = kbd;
        for (int g = 0; g < 8; ++g) {
            gp.kb_off[g] = c->kb_l2l_off[g];
            gp.kb_cnt[g] = 1;
        }
        gp.n_src = 1 << l;
        gp.n_tgt = 1 << (l + 1);
        gp.mode = 2;
        gp.grouped = 1;
        gp.accumulate = 1;
        gp.pc = c->pc;
        if ((rc = launch_gemm(c, gp, 8, (int64_t)1 << (3 * l)))) return rc;
    }
    return VFMM_OK;
}

int check_device_error(Ctx *c)
{
    int e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "device sync");
    if (e) {
        cudaMemsetAsync(c->err.p, 0, sizeof(int), c->stream);
        if (e & ERRBIT_LEAF_OVERFLOW)
            return fail(c, VFMM_ERR_UNSUPPORTED, "a leaf holds more particles than the per-leaf sort capacity (4096); use a deeper tree");
        if (e & ERRBIT_TIMEOUT) return fail(c, VFMM_ERR_TIMEOUT, "a bounded device wait gave up");
        if (e & ERRBIT_NONFINITE) return fail(c, VFMM_ERR_ARG, "a position is NaN or infinite");
        return fail(c, VFMM_ERR_BOUNDS, "a device bounds check fired");
    }
    return VFMM_OK;
}

// near_only (with grad): the near-field P2P alone, no far field (the adjoint adds the
// transposed far field itself)
int eval_impl(Ctx *c, const void *gamma, double sigma, void *u_out, void *s_out, bool grad = false,
              bool near_only = false)
{
    if (!c->built) return fail(c, VFMM_ERR_NOT_BUILT, "vfmm_build_tree has not been called");
    if (!gamma || !u_out) return fail(c, VFMM_ERR_ARG, "null gamma or u_out");
    if (!std::isfinite(sigma) || sigma <= 0.0) return fail(c, VFMM_ERR_ARG, "sigma must be finite and > 0");
    const bool fmm = c->cfg.method == VFMM_METHOD_FMM;
    // Every pair closer than rho_cut sigma takes the smoothed kernel: Rreq rings of leaves
    // cover them.  The FP32 velocity / stretching path keeps one ring in the near field and
    // gives the second ring to the M2L, adding there the smoothed-minus-singular correction
    // for the source octants that come within rho_cut sigma; FP64 and the gradient path
    // take all Rreq rings in the near field.
    int R, Rc = 0;
    if (fmm) {
        int Rreq = 1;
        while (Rreq * c->leaf_w < c->cfg.rho_cut * sigma && Rreq < 3) ++Rreq;
        if (Rreq > 2)
            return fail(c, VFMM_ERR_UNSUPPORTED,
                        "the near field would need more than 2 rings of leaves (rho_cut * sigma > 2 * leaf width); use a shallower tree");
        const bool corr_ok = !c->f64 && !grad;
        R = c->cfg.near_rings > 0 ? c->cfg.near_rings : (corr_ok ? 1 : Rreq);
        if (corr_ok && Rreq > R) Rc = Rreq;
    } else {
        R = c->cfg.direct_images;
    }
    c->last_R = R;
    c->last_Rc = Rc;
    cudaStream_t main_st = c->stream;
    int rc;
    cudaEventRecord(c->ev[2], main_st);
    if ((rc = launch_gather_gamma(c, gamma))) return rc;
    const void *uf = nullptr, *sf = nullptr;
    // FP32 velocity / stretching: the far field runs on a high-priority side stream while the
    // P2P (near field only) runs on the caller's stream; a last kernel adds the far field
    const bool overlap = fmm && !grad && !c->f64 && c->overlap && c->side;
    // fork onto the side stream; with VFMM_FORK_AT_M2L the upward pass (P2M, M2M, root: FP32
    // ALU work like the P2P's) runs in line first and only the M2L (tensor cores) and the
    // downward pass run beside the P2P
    auto fork = [&]() {
        cudaEventRecord(c->ev[11], main_st);
        cudaStreamWaitEvent(c->side, c->ev[11], 0);
        c->stream = c->side;
    };
    if (overlap && !VFMM_FORK_AT_M2L) fork();
    cudaStream_t st = c->stream;
    struct Restore {
        Ctx *c;
        cudaStream_t s;
        ~Restore() { c->stream = s; }
    } restore{c, main_st};
    if (fmm && !near_only) {
        const int D = c->depth;
        const int S = c->cfg.periodic_levels;
        const int4 *kbd = (const int4 *)c->kblocks.p;
        char *M = (char *)c->mexp.p, *L = (char *)c->lexp.p;
        auto lvl = [&](char *base, int l) { return (void *)(base + c->lvl_off[l] * c->esz); };
        if ((rc = launch_p2m(c))) return rc;
        cudaEventRecord(c->ev[3], st);
        for (int l = D - 1; l >= 1; --l) {
            GemmParams gp = {};
            gp.AT = c->at_m2m.p;
            gp.B = lvl(M, l + 1);
            gp.C = lvl(M, l);
            gp.kb = kbd;
            gp.kb_off[0] = c->kb_m2m_off;
            gp.kb_cnt[0] = 8;
            gp.n_src = 1 << (l + 1);
            gp.n_tgt = 1 << l;
            gp.mode = 1;
            gp.grouped = 0;
            gp.accumulate = 0;
            gp.pc = c->pc;
            if ((rc = launch_gemm(c, gp, 1, (int64_t)1 << (3 * l)))) return rc;
        }
        cudaEventRecord(c->ev[4], st);
        if (S > 0) {
            if ((rc = launch_root(c))) return rc;
        }
        cudaEventRecord(c->ev[5], st);
        const bool tc = c->cfg.m2l_prec == VFMM_M2L_TF32X3 || c->cfg.m2l_prec == VFMM_M2L_BF16X3;
        bool presplit = false;  // the leaf level's hi/lo split already issued
        if (overlap && VFMM_FORK_AT_M2L) {
            // the leaf split in line, so that the first far-field launch beside the P2P is the
            // leaf M2L itself
            if (tc && VFMM_M2L_LEAF_FIRST && D >= 3) {
                if ((rc = launch_split(c, D, c->cfg.m2l_prec == VFMM_M2L_BF16X3))) return rc;
                presplit = true;
            }
            fork();
            st = c->stream;
        }
        // the levels' M2L are independent; VFMM_M2L_LEAF_FIRST issues the leaf level first
        for (int li = 0; li < D; ++li) {
            const int l = VFMM_M2L_LEAF_FIRST ? D - li : li + 1;
            int Rl = (l == D) ? R : 1;
            if (tc && l >= VFMM_TC_MIN_LEVEL) {
                bool bf = c->cfg.m2l_prec == VFMM_M2L_BF16X3;
                if (!(presplit && l == D) && (rc = launch_split(c, l, bf))) return rc;
                if ((rc = launch_tc_m2l(c, l, Rl, bf))) return rc;
                continue;
            }
            GemmParams gp = {};
            gp.AT = c->at_m2l.p;
            gp.B = lvl(M, l);
            gp.C = lvl(L, l);
            gp.kb = kbd;
            for (int g = 0; g < 8; ++g) {
                gp.kb_off[g] = c->kb_m2l_off[Rl][g];
                gp.kb_cnt[g] = c->kb_m2l_cnt[Rl][g];
            }
            gp.n_src = gp.n_tgt = 1 << l;
            gp.mode = 0;
            gp.grouped = 1;
            gp.accumulate = 0;
            gp.pc = c->pc;
            if ((rc = launch_gemm(c, gp, 8, (int64_t)1 << (3 * (l - 1))))) return rc;
        }
        cudaEventRecord(c->ev[6], st);
        for (int l = 1; l <= D; ++l) {
            if (l == 1 && S == 0) continue;
            GemmParams gp = {};
            gp.AT = c->at_l2l.p;
            gp.B = lvl(L, l - 1);
            gp.C = lvl(L, l);
            gp.kb = kbd;
            for (int g = 0; g < 8; ++g) {
                gp.kb_off[g] = c->kb_l2l_off[g];
                gp.kb_cnt[g] = 1;
            }
            gp.n_src = 1 << (l - 1);
            gp.n_tgt = 1 << l;
            gp.mode = 2;
            gp.grouped = 1;
            gp.accumulate = 1;
            gp.pc = c->pc;
            if ((rc = launch_gemm(c, gp, 8, (int64_t)1 << (3 * (l - 1))))) return rc;
        }
        cudaEventRecord(c->ev[7], st);
        if ((rc = launch_l2p(c, grad))) return rc;
        cudaEventRecord(c->ev[10], st);
        uf = c->ufar.p;
        sf = grad ? c->gfar.p : c->sfar.p;
    } else {
        for (int k = 3; k <= 7; ++k) cudaEventRecord(c->ev[k], st);
        cudaEventRecord(c->ev[10], st);
    }
    c->stream = main_st;
    cudaEventRecord(c->ev[8], main_st);
    if (grad) {
        if ((rc = launch_p2p_grad(c, R, sigma, uf, sf, u_out, s_out, fmm ? -1 : c->cfg.direct_images))) return rc;
    } else if (overlap) {
        c->p2p_shared_blocks = VFMM_P2P_SHARED_BLOCKS;
        rc = launch_p2p(c, R, Rc, sigma, nullptr, nullptr, u_out, s_out, -1);
        c->p2p_shared_blocks = 0;
        if (rc) return rc;
    } else {
        if ((rc = launch_p2p(c, R, Rc, sigma, uf, sf, u_out, s_out, fmm ? -1 : c->cfg.direct_images))) return rc;
    }
    cudaEventRecord(c->ev[9], main_st);
    if (overlap) {
        cudaStreamWaitEvent(main_st, c->ev[10], 0);
        if ((rc = launch_add_far(c, u_out, s_out))) return rc;
    }
    c->timed_eval = true;
    return VFMM_OK;
}

int build_impl(Ctx *c, int64_t n, const void *x, double sigma_hint = 0.0)
{
    if (n <= 0) return fail(c, VFMM_ERR_ARG, "n must be > 0");
    if (n > (int64_t)1 << 30) return fail(c, VFMM_ERR_UNSUPPORTED, "n above 2^30 particles");
    if (!x) return fail(c, VFMM_ERR_ARG, "null x");
    int D;
    if (c->depth_override >= 0) {
        D = c->depth_override;
    } else if (c->cfg.depth > 0) {
        D = c->cfg.depth;
    } else {
        double ratio = (double)n / (double)(c->cfg.ncrit > 0 ? c->cfg.ncrit : 64);
        D = (int)std::lround(std::log(ratio > 1.0 ? ratio : 1.0) / std::log(8.0));
        if (D < 1) D = 1;
        if (D > MAX_DEPTH) D = MAX_DEPTH;
        // a known core size (time stepping with core spreading): the shallowest change of
        // depth that keeps the near field within two rings, 2 w >= rho_cut sigma
        if (sigma_hint > 0.0 && c->cfg.method == VFMM_METHOD_FMM && c->cfg.near_rings == 0)
            while (D > 1 && 2.0 * (c->cfg.box / (1 << D)) < c->cfg.rho_cut * sigma_hint) --D;
    }
    c->depth = D;
    c->nside = 1 << D;
    c->nleaf = (int64_t)1 << (3 * D);
    c->leaf_w = c->cfg.box / c->nside;
    c->n = n;
    c->built = false;
    const size_t esz = c->esz;
    int st;
    if ((st = ensure(c, c->xs, (size_t)n * 4 * esz, "positions"))) return st;
    if ((st = ensure(c, c->gs, (size_t)n * 4 * esz, "strengths"))) return st;
    if ((st = ensure(c, c->perm, (size_t)n * sizeof(int), "permutation"))) return st;
    if ((st = ensure(c, c->keys, (size_t)n * sizeof(int), "keys"))) return st;
    if ((st = ensure(c, c->tmpidx, (size_t)n * sizeof(int), "scatter"))) return st;
    if ((st = ensure(c, c->counts, (size_t)c->nleaf * sizeof(int), "counts"))) return st;
    if ((st = ensure(c, c->fill, (size_t)c->nleaf * sizeof(int), "fill"))) return st;
    if ((st = ensure(c, c->leaf_start, (size_t)(c->nleaf + 1) * sizeof(int), "leaf ranges"))) return st;
    if ((st = ensure(c, c->scan_part, (size_t)((c->nleaf + 1023) / 1024 + 1) * sizeof(int), "scan"))) return st;
    if ((st = ensure(c, c->maxleaf, sizeof(int), "max leaf"))) return st;
    if ((st = ensure(c, c->bbox, (size_t)c->nleaf * 2 * sizeof(float4), "leaf boxes"))) return st;
    if ((st = ensure(c, c->oct_start, (size_t)c->nleaf * 8 * sizeof(int), "octant starts"))) return st;
    if ((st = ensure(c, c->oct_box, (size_t)c->nleaf * 16 * sizeof(float4), "octant boxes"))) return st;
    if (c->cfg.method == VFMM_METHOD_FMM) {
        c->lvl_off.assign(D + 2, 0);
        size_t tot = 0;
        for (int l = 0; l <= D; ++l) {
            c->lvl_off[l] = tot;
            tot += ((size_t)1 << (3 * l)) * 3 * c->pc;
        }
        c->lvl_off[D + 1] = tot;
        if ((st = ensure(c, c->mexp, tot * esz, "multipoles"))) return st;
        if ((st = ensure(c, c->lexp, tot * esz, "locals"))) return st;
        if ((st = ensure(c, c->ufar, (size_t)n * 3 * esz, "far velocity"))) return st;
        if (c->cfg.m2l_prec == VFMM_M2L_TF32X3 || c->cfg.m2l_prec == VFMM_M2L_BF16X3) {
            size_t cnt = 0;
            for (int l = 3; l <= D; ++l) cnt = std::max(cnt, split_count(l, c->pc));
            size_t eb = c->cfg.m2l_prec == VFMM_M2L_BF16X3 ? 2 : 4;
            if ((st = ensure(c, c->mhi, cnt * eb, "multipole hi"))) return st;
            if ((st = ensure(c, c->mlo, cnt * eb, "multipole lo"))) return st;
        }
        if ((st = ensure(c, c->sfar, (size_t)n * 3 * esz, "far stretching"))) return st;
        if ((st = ensure(c, c->gemm_part, (size_t)64 << 20, "split-k partials"))) return st;
    }
    c->launches = 0;
    cudaEventRecord(c->ev[0], c->stream);
    // keys, counts and the scatter into leaves; the largest leaf sizes the per-leaf sort
    if ((st = launch_tree(c, x))) return st;
    int ml = 0;
    cudaError_t e = cudaMemcpyAsync(&ml, c->maxleaf.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read leaf occupancy");
    if ((st = check_device_error(c))) return st;
    c->max_leaf = ml;
    if (ml > LEAF_SORT_CAP)
        return fail(c, VFMM_ERR_UNSUPPORTED, "a leaf holds more particles than the per-leaf sort capacity (4096); use a deeper tree");
    if ((st = launch_leaf_sort(c, x, ml))) return st;
    cudaEventRecord(c->ev[1], c->stream);
    // no second synchronisation: the leaf sort can only raise the checked build's bounds bit
    // (the largest leaf was checked above), which vfmm_sync reports like any evaluation error;
    // the caller can queue the evaluation while the sort runs
    c->built = true;
    return VFMM_OK;
}

}  // namespace

extern "C" {

int vfmm_config_default(vfmm_config *cfg)
{
    if (!cfg) return VFMM_ERR_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->p = 10;
    cfg->depth = 0;
    cfg->ncrit = 64;
    cfg->near_rings = 0;
    cfg->rho_cut = 5.0;
    cfg->concurrent_far = 1;
    cfg->periodic_levels = 2;
    cfg->box = 6.283185307179586477;
    cfg->dtype = VFMM_F32;
    cfg->m2l_prec = VFMM_M2L_BF16X3;
    cfg->method = VFMM_METHOD_FMM;
    cfg->direct_images = 1;
    cfg->stream = nullptr;
    return VFMM_OK;
}

int vfmm_create(const vfmm_config *cfg, vfmm_handle *out)
{
    if (!out) return VFMM_ERR_ARG;
    *out = nullptr;
    if (!cfg) return VFMM_ERR_ARG;
    const vfmm_config &k = *cfg;
    if (k.dtype != VFMM_F32 && k.dtype != VFMM_F64) return VFMM_ERR_ARG;
    if (k.method != VFMM_METHOD_FMM && k.method != VFMM_METHOD_DIRECT) return VFMM_ERR_ARG;
    if (!(k.box > 0.0) || !std::isfinite(k.box)) return VFMM_ERR_ARG;
    if (k.depth < 0 || k.depth > MAX_DEPTH) return VFMM_ERR_ARG;
    if (k.method == VFMM_METHOD_FMM) {
        if (k.p < 2) return VFMM_ERR_ARG;
        if ((k.p + 1) * (k.p + 1) > OUT_ROWS) return VFMM_ERR_UNSUPPORTED;
        if (k.periodic_levels < 0 || k.periodic_levels > 8) return VFMM_ERR_ARG;
        if (k.depth < 0 || k.depth > MAX_DEPTH) return VFMM_ERR_ARG;
        if (k.near_rings < 0 || k.near_rings > 2) return VFMM_ERR_UNSUPPORTED;
        if (!(k.rho_cut > 0.0)) return VFMM_ERR_ARG;
        if (k.m2l_prec < VFMM_M2L_FP32 || k.m2l_prec > VFMM_M2L_BF16X3) return VFMM_ERR_ARG;
        if (k.dtype == VFMM_F64 && k.m2l_prec != VFMM_M2L_FP64) return VFMM_ERR_ARG;
        if (k.dtype == VFMM_F32 && k.m2l_prec == VFMM_M2L_FP64) return VFMM_ERR_ARG;
    } else {
        if (k.direct_images < 0 || k.direct_images > 20) return VFMM_ERR_ARG;
    }
    vfmm_ctx *h = new (std::nothrow) vfmm_ctx;
    if (!h) return VFMM_ERR_OOM;
    Ctx *c = &h->c;
    c->cfg = k;
    c->stream = (cudaStream_t)k.stream;
    c->overlap = k.concurrent_far != 0;
    c->f64 = k.dtype == VFMM_F64;
    c->esz = c->f64 ? 8 : 4;
    c->p = k.method == VFMM_METHOD_FMM ? k.p : 2;
    c->nc = (c->p + 1) * (c->p + 1);
    c->pc = ((c->nc + 31) / 32) * 32;
    for (int i = 0; i < 12; ++i) {
        if (cudaEventCreate(&c->ev[i]) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) cudaEventDestroy(c->ev[j]);
            delete h;
            return VFMM_ERR_CUDA;
        }
    }
    c->have_events = true;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            c->sm_count = sms;
        cudaGetLastError();
    }
    {
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi) != cudaSuccess) {
            cudaGetLastError();
            c->side = nullptr;  // the far field then runs in line with the P2P
        }
    }
    int st = ensure(c, c->err, sizeof(int), "error word");
    if (!st && cudaMemset(c->err.p, 0, sizeof(int)) != cudaSuccess) st = VFMM_ERR_CUDA;
    if (!st && k.method == VFMM_METHOD_FMM) {
        set_constants(c->p);
        st = c->f64 ? build_operators<double>(c) : build_operators<float>(c);
    }
    if (st) {
        vfmm_destroy(h);
        return st;
    }
    *out = h;
    return VFMM_OK;
}

int vfmm_destroy(vfmm_handle h)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->xs, &c->gs, &c->perm, &c->keys, &c->leaf_start, &c->counts, &c->fill, &c->tmpidx,
                      &c->scan_part, &c->err, &c->maxleaf, &c->bbox, &c->oct_start, &c->oct_box, &c->mexp, &c->lexp, &c->mhi, &c->mlo, &c->gemm_part, &c->ufar,
                      &c->sfar, &c->gfar, &c->adj_u, &c->adj_g1, &c->adj_g2, &c->rk_u1, &c->rk_s1, &c->rk_u2, &c->rk_s2, &c->rk_x1, &c->rk_g1, &c->diag, &c->rg_om, &c->rg_r, &c->rg_d, &c->rg_q, &c->rg_t1, &c->rg_t2, &c->rg_dots, &c->at_m2l, &c->at_m2m, &c->at_l2l, &c->tc_hi, &c->tc_lo, &c->at_m2l_t, &c->at_m2m_t, &c->at_l2l_t, &c->tc_hi_t, &c->tc_lo_t, &c->m2m_f64,
                      &c->lattice_f64, &c->root_m, &c->kblocks, &c->cls, &c->spec_work, &c->spec_E, &c->hx, &c->hg, &c->hu, &c->hs};
    for (DevBuf *b : bufs) release(*b);
    if (c->have_events)
        for (int i = 0; i < 12; ++i) cudaEventDestroy(c->ev[i]);
    if (c->side) cudaStreamDestroy(c->side);
    delete h;
    return VFMM_OK;
}

int vfmm_set_stream(vfmm_handle h, void *stream)
{
    if (!h) return VFMM_ERR_ARG;
    h->c.stream = (cudaStream_t)stream;
    h->c.cfg.stream = stream;
    return VFMM_OK;
}

int vfmm_set_wait_limit(vfmm_handle h, int64_t tries)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (tries < 0) return fail(c, VFMM_ERR_ARG, "tries must be >= 0");
    c->wait_limit = tries > 0 ? (long long)tries : (1LL << 26);
    return VFMM_OK;
}

int vfmm_build_tree(vfmm_handle h, int64_t n, const void *x)
{
    if (!h) return VFMM_ERR_ARG;
    return build_impl(&h->c, n, x);
}

int vfmm_eval_velocity_stretching(vfmm_handle h, const void *gamma, double sigma, void *u_out, void *s_out)
{
    if (!h) return VFMM_ERR_ARG;
    return eval_impl(&h->c, gamma, sigma, u_out, s_out);
}

int vfmm_eval_velocity_gradient(vfmm_handle h, const void *gamma, double sigma, void *u_out, void *g_out)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (!g_out) return fail(c, VFMM_ERR_ARG, "null g_out");
    if (c->built && c->cfg.method == VFMM_METHOD_FMM) {
        int st = ensure(c, c->gfar, (size_t)c->n * 9 * c->esz, "far velocity gradient");
        if (st) return st;
    }
    return eval_impl(c, gamma, sigma, u_out, g_out, true);
}

int vfmm_eval_adjoint(vfmm_handle h, const void *gamma, double sigma, const void *w, const void *v, void *dgamma,
                      void *dx)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (v) return fail(c, VFMM_ERR_UNSUPPORTED, "a loss through the stretching term (v != NULL) is not supported");
    if (!w || !dgamma || !dx || !gamma) return fail(c, VFMM_ERR_ARG, "null argument");
    if (!c->built) return fail(c, VFMM_ERR_NOT_BUILT, "vfmm_build_tree has not been called");
    size_t n = (size_t)c->n;
    int st;
    if ((st = ensure(c, c->adj_u, n * 3 * c->esz, "adjoint velocity"))) return st;
    if ((st = ensure(c, c->adj_g1, n * 9 * c->esz, "adjoint gradient"))) return st;
    if ((st = ensure(c, c->adj_g2, n * 9 * c->esz, "adjoint gradient"))) return st;
    if (c->cfg.method != VFMM_METHOD_FMM) {
        // direct sum: grad u of the gamma field, then velocity and grad u of the w field
        // (dL/dgamma = A w, A symmetric)
        if ((st = vfmm_eval_velocity_gradient(h, gamma, sigma, c->adj_u.p, c->adj_g1.p))) return st;
        if ((st = vfmm_eval_velocity_gradient(h, w, sigma, dgamma, c->adj_g2.p))) return st;
        return launch_adjoint_combine(c, c->adj_g1.p, w, c->adj_g2.p, gamma, nullptr, dx);
    }
    // FMM: the exact transpose of the evaluated operator.  (1) grad u of the gamma field (near
    // and far: the target-position term); (2) the near field of w (symmetric pair set: its
    // velocity is the near part of A^T w, its gradient gives the near source-position term);
    // (3) the transposed far field of w adds P^T ... E^T w to dgamma and writes the far
    // source-position term; (4) dx = G1^T w + G2_near^T gamma + far term.
    if (!c->have_transposed) {
        st = c->f64 ? build_transposed<double>(c) : build_transposed<float>(c);
        if (st) return st;
    }
    if ((st = vfmm_eval_velocity_gradient(h, gamma, sigma, c->adj_u.p, c->adj_g1.p))) return st;
    if ((st = eval_impl(c, w, sigma, dgamma, c->adj_g2.p, true, true))) return st;
    if ((st = far_transpose(c, c->last_R))) return st;
    if ((st = launch_dual_l2p(c, gamma, dgamma, c->adj_u.p))) return st;
    return launch_adjoint_combine(c, c->adj_g1.p, w, c->adj_g2.p, gamma, c->adj_u.p, dx);
}

int vfmm_rk_step(vfmm_handle h, int64_t n, void *x, void *gamma, double *sigma, double dt, double nu)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (n <= 0 || !x || !gamma || !sigma) return fail(c, VFMM_ERR_ARG, "bad arguments");
    if (!std::isfinite(dt) || !std::isfinite(nu) || nu < 0.0) return fail(c, VFMM_ERR_ARG, "dt and nu must be finite, nu >= 0");
    const double s0 = *sigma;
    if (!std::isfinite(s0) || s0 <= 0.0) return fail(c, VFMM_ERR_ARG, "sigma must be finite and > 0");
    const double s1sq = s0 * s0 + 2.0 * nu * dt;
    if (!(s1sq > 0.0)) return fail(c, VFMM_ERR_ARG, "sigma^2 + 2 nu dt must be > 0");
    const double s1 = std::sqrt(s1sq);
    const size_t bytes = (size_t)n * 3 * c->esz;
    int st;
    DevBuf *tmp[] = {&c->rk_u1, &c->rk_s1, &c->rk_u2, &c->rk_s2, &c->rk_x1, &c->rk_g1};
    for (DevBuf *b : tmp)
        if ((st = ensure(c, *b, bytes, "time-step temporaries"))) return st;
    const double L = c->cfg.box;
    // stage 1 at (x, gamma, sigma)
    if ((st = build_impl(c, n, x, s0))) return st;
    if ((st = eval_impl(c, gamma, s0, c->rk_u1.p, c->rk_s1.p))) return st;
    if ((st = launch_axpy3(c, n, x, c->rk_u1.p, nullptr, dt, L, c->rk_x1.p))) return st;
    if ((st = launch_axpy3(c, n, gamma, c->rk_s1.p, nullptr, dt, 0.0, c->rk_g1.p))) return st;
    // stage 2 at (x + dt u1, gamma + dt S1, sqrt(sigma^2 + 2 nu dt))
    if ((st = build_impl(c, n, c->rk_x1.p, s1))) return st;
    if ((st = eval_impl(c, c->rk_g1.p, s1, c->rk_u2.p, c->rk_s2.p))) return st;
    if ((st = launch_axpy3(c, n, x, c->rk_u1.p, c->rk_u2.p, 0.5 * dt, L, x))) return st;
    if ((st = launch_axpy3(c, n, gamma, c->rk_s1.p, c->rk_s2.p, 0.5 * dt, 0.0, gamma))) return st;
    *sigma = s1;
    c->built = false;  // the tree holds the stage-2 positions
    return VFMM_OK;
}

int vfmm_reinit(vfmm_handle h, int64_t n, const void *x, const void *gamma, double sigma, int m, double sigma_new,
                int iters, void *x_new, void *gamma_new, double *residual)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (n <= 0 || !x || !gamma || !x_new || !gamma_new) return fail(c, VFMM_ERR_ARG, "bad arguments");
    if (m < 2 || (int64_t)m * m * m > ((int64_t)1 << 30)) return fail(c, VFMM_ERR_ARG, "lattice size m out of range");
    if (iters < 0 || iters > 100000) return fail(c, VFMM_ERR_ARG, "iters out of range");
    if (!std::isfinite(sigma) || sigma <= 0.0) return fail(c, VFMM_ERR_ARG, "sigma must be finite and > 0");
    const double hl = c->cfg.box / m;
    if (!(sigma_new > 0.0)) sigma_new = hl;
    if (!std::isfinite(sigma_new)) return fail(c, VFMM_ERR_ARG, "sigma_new must be finite");
    // octree of the old particles with leaves aligned to the new lattice (m divisible by 2^D)
    double ratio = (double)n / (double)(c->cfg.ncrit > 0 ? c->cfg.ncrit : 64);
    int D = (int)std::lround(std::log(ratio > 1.0 ? ratio : 1.0) / std::log(8.0));
    if (D > MAX_DEPTH) D = MAX_DEPTH;
    while (D > 0 && (m % (1 << D)) != 0) --D;
    if ((m >> D) > 64) return fail(c, VFMM_ERR_UNSUPPORTED, "lattice too fine for the particle tree");
    c->depth_override = D;
    int st = build_impl(c, n, x);
    c->depth_override = -1;
    if (st) return st;
    if ((st = launch_gather_gamma(c, gamma))) return st;
    int R = (int)std::ceil(6.0 * sigma / c->leaf_w);
    if (R < 1) R = 1;
    const size_t bytes = (size_t)m * m * m * 3 * c->esz;
    DevBuf *tmp[] = {&c->rg_om, &c->rg_r, &c->rg_d, &c->rg_q, &c->rg_t1, &c->rg_t2};
    for (DevBuf *b : tmp)
        if ((st = ensure(c, *b, bytes, "reinitialisation temporaries"))) return st;
    if ((st = ensure(c, c->rg_dots, 4 * sizeof(double), "reinitialisation sums"))) return st;
    st = launch_reinit(c, m, sigma, sigma_new, iters, R, x_new, gamma_new, residual);
    c->built = false;  // the tree holds the old particles
    return st;
}

int vfmm_diagnostics(vfmm_handle h, int64_t n, const void *x, const void *gamma, const void *u, double *out)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (n <= 0 || !x || !gamma || !out) return fail(c, VFMM_ERR_ARG, "bad arguments");
    int st;
    if ((st = ensure(c, c->diag, 8 * sizeof(double), "diagnostics"))) return st;
    cudaMemsetAsync(c->diag.p, 0, 8 * sizeof(double), c->stream);
    if ((st = launch_diag(c, n, x, gamma, u, (double *)c->diag.p))) return st;
    cudaError_t e = cudaMemcpyAsync(out, c->diag.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics");
    return VFMM_OK;
}

int vfmm_energy_spectrum(vfmm_handle h, int n, const void *u_lattice, int kmax, double *E_out)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (!u_lattice || !E_out) return fail(c, VFMM_ERR_ARG, "null u_lattice or E_out");
    if (n < 4 || n > 1024 || (n & (n - 1))) return fail(c, VFMM_ERR_UNSUPPORTED, "n must be a power of two in [4, 1024]");
    if (kmax < 0 || kmax > 4096) return fail(c, VFMM_ERR_ARG, "kmax must be in [0, 4096]");
    const size_t m = (size_t)n * n * n;
    int st;
    if ((st = ensure(c, c->spec_work, 3 * m * sizeof(double2), "spectrum workspace"))) return st;
    if ((st = ensure(c, c->spec_E, (size_t)(kmax + 1) * sizeof(double), "spectrum shells"))) return st;
    if ((st = launch_spectrum(c, n, u_lattice, kmax, (double2 *)c->spec_work.p, (double *)c->spec_E.p))) return st;
    cudaError_t e = cudaMemcpyAsync(E_out, c->spec_E.p, (size_t)(kmax + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "energy spectrum");
    return VFMM_OK;
}

int vfmm_derivative_moments(vfmm_handle h, int64_t n, const void *grad, double *out)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (n <= 0 || !grad || !out) return fail(c, VFMM_ERR_ARG, "bad arguments");
    int st;
    if ((st = ensure(c, c->diag, 8 * sizeof(double), "diagnostics"))) return st;
    cudaMemsetAsync(c->diag.p, 0, 3 * sizeof(double), c->stream);
    if ((st = launch_moments(c, n, grad, (double *)c->diag.p))) return st;
    double s[3];
    cudaError_t e = cudaMemcpyAsync(s, c->diag.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "derivative moments");
    const double cnt = 3.0 * (double)n;
    out[0] = s[0] / cnt;
    out[1] = s[1] / cnt;
    out[2] = s[2] / cnt;
    out[3] = out[1] / std::pow(out[0], 1.5);
    out[4] = out[2] / (out[0] * out[0]);
    return VFMM_OK;
}

int vfmm_eval_host(vfmm_handle h, int64_t n, const void *x, const void *gamma, double sigma, void *u_out,
                   void *s_out)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (n <= 0 || !x || !gamma || !u_out) return fail(c, VFMM_ERR_ARG, "bad host arguments");
    size_t bytes = (size_t)n * 3 * c->esz;
    int st;
    if ((st = ensure(c, c->hx, bytes, "host staging x"))) return st;
    if ((st = ensure(c, c->hg, bytes, "host staging gamma"))) return st;
    if ((st = ensure(c, c->hu, bytes, "host staging u"))) return st;
    if ((st = ensure(c, c->hs, bytes, "host staging S"))) return st;
    // x on the caller's stream (the tree needs it first); gamma on the side stream, so its copy
    // runs while the tree is built, joined before the evaluation
    cudaError_t e = cudaMemcpyAsync(c->hx.p, x, bytes, cudaMemcpyHostToDevice, c->stream);
    const bool side_copy = c->side != nullptr;
    if (e == cudaSuccess && side_copy) {
        cudaEventRecord(c->ev[11], c->stream);  // the side stream follows earlier work on the caller's
        cudaStreamWaitEvent(c->side, c->ev[11], 0);
        e = cudaMemcpyAsync(c->hg.p, gamma, bytes, cudaMemcpyHostToDevice, c->side);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev[10], c->side);
    } else if (e == cudaSuccess) {
        e = cudaMemcpyAsync(c->hg.p, gamma, bytes, cudaMemcpyHostToDevice, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "host to device copy");
    if ((st = build_impl(c, n, c->hx.p))) return st;
    if (side_copy) cudaStreamWaitEvent(c->stream, c->ev[10], 0);
    if ((st = eval_impl(c, c->hg.p, sigma, c->hu.p, s_out ? c->hs.p : nullptr))) return st;
    e = cudaMemcpyAsync(u_out, c->hu.p, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && s_out) e = cudaMemcpyAsync(s_out, c->hs.p, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device to host copy");
    return check_device_error(c);
}

int vfmm_sync(vfmm_handle h)
{
    if (!h) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    int st = check_device_error(c);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "asynchronous CUDA error");
    return VFMM_OK;
}

int vfmm_get_timings(vfmm_handle h, double *ms, int nphase)
{
    if (!h || !ms || nphase < 0) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    if (!c->timed_eval) return fail(c, VFMM_ERR_NOT_BUILT, "no evaluation has been timed");
    // L2P ends at [10]; with the far field on the side stream the phases overlap the P2P
    const int pairs[8][2] = {{0, 1}, {2, 3}, {3, 4}, {5, 6}, {4, 5}, {6, 7}, {7, 10}, {8, 9}};
    for (int i = 0; i < nphase && i < NPHASE; ++i) {
        float t = 0.f;
        cudaError_t e = cudaEventElapsedTime(&t, c->ev[pairs[i][0]], c->ev[pairs[i][1]]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            t = 0.f;
        }
        ms[i] = t;
    }
    return VFMM_OK;
}

int vfmm_get_tree_info(vfmm_handle h, int64_t *out, int nout)
{
    if (!h || !out) return VFMM_ERR_ARG;
    Ctx *c = &h->c;
    int64_t pairs = 0;
    if (VFMM_CHECK && nout > 7) {
        cudaStreamSynchronize(c->stream);
        pairs = p2p_pairs_read();
    }
    int64_t v[8] = {c->depth, c->last_R, c->nside, c->max_leaf, c->n, c->launches, c->last_Rc, pairs};
    for (int i = 0; i < nout && i < 8; ++i) out[i] = v[i];
    return VFMM_OK;
}

const char *vfmm_strerror(int status)
{
    switch (status) {
    case VFMM_OK: return "ok";
    case VFMM_ERR_ARG: return "invalid argument";
    case VFMM_ERR_CUDA: return "CUDA error";
    case VFMM_ERR_OOM: return "out of device memory";
    case VFMM_ERR_NOT_BUILT: return "tree not built";
    case VFMM_ERR_BOUNDS: return "device bounds check";
    case VFMM_ERR_TIMEOUT: return "device wait timed out";
    case VFMM_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

const char *vfmm_last_error(vfmm_handle h)
{
    if (!h) return "null handle";
    return h->c.last_error.c_str();
}

}  // extern "C"

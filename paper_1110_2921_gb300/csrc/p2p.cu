// Near-field P2P of the Gaussian-regularised Biot-Savart kernel and its stretching term.
//
// For every target i and every source j in the (2R+1)^3 neighbour leaves of i's leaf
// (periodically wrapped, each with its image shift), excluding j = i:
//   u_i += K(r) gamma_j x r,                         Eq. (biotsavart)
//   S_i += K(r) gamma_j x gamma_i + F(r)(gamma_i.r)(gamma_j x r)      Eq. (stretching)
//   K = q(rho)/(4 pi r^3),  F = K'(r)/r,  q from Eq. (cutoff).
// The near field is "solved exactly" (Section 3.1): the full smoothed kernel, no expansion.
//
// FP32 kernel (k_p2p_f32): one warp per target leaf (and 64-target chunk), two targets per
// lane.  The sources of each neighbour leaf are staged in shared memory as (x, gamma,
// gamma x x) records relative to the target leaf centre (the image shift applied once per
// leaf) and read as warp-wide broadcasts.  Per target four accumulated vectors,
//   A = sum K gamma_j,  U = sum K (gamma_j x x_j),  D = sum f gamma_j,  E = sum f (gamma_j x x_j),
// f = F (gamma_i . r), give u = A x x_i - U and S = A x gamma_i + D x x_i - E without a cross
// product per pair.  The inner loop is chosen per run of source octants by the gap between
// the target leaf's box and the octant's box: smoothed with the small-rho series branch,
// smoothed, singular (gap >= 6.5 sigma), or, in ring 2 beyond the near ring, smoothed minus
// singular for octants within rho_cut sigma (the Gaussian tail the far field lacks).
// FP32 math:
//   * 1/r from rsqrt, exp(-rho^2/2) from ex2 on coordinates pre-scaled by
//     sqrt(log2 e / (2 sigma^2)), both single MUFU instructions;
//   * erf(rho/sqrt2) by Abramowitz & Stegun 7.1.26 (Hastings' rational approximation,
//     |error| <= 1.5e-7), which needs exactly the exp(-rho^2/2) already computed;
//   * for rho < 0.5 the Taylor series of q/rho^3 and of K'/r in rho^2, which avoids the
//     cancellation of q ~ rho^3 and the 1/r^5 of F, and gives the exact self-pair limit
//     (K finite, r = 0 so every self term vanishes).
// The epilogue scatters u, S to caller order, adding the far field when it is given (in line);
// with the concurrent far field, k_add_far adds it afterwards.  k_p2p_f64 (FP64 near field),
// k_p2p_grad (velocity gradient for the adjoint) and the allocation-free direct sum at the end
// of the file use one thread per target.
#include "common.cuh"
#include "vfmm_internal.h"

#include <algorithm>
#include <cmath>

namespace vfmm {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct P2PConst {
    double sigma, L;
    // FP32 constants (folded sigma factors)
    float ce;      // -log2(e) / (2 sigma^2): exp(-rho^2/2) = 2^(r2 * ce)
    float ct;      // 0.3275911 / (sqrt2 sigma): A&S t = 1/(1 + ct r)
    float cq;      // sqrt(2/pi) / sigma
    float cf;      // sqrt(2/pi) / sigma^3
    float zs;      // series threshold on r2 * ce (rho < 0.5)
    float inv_s2;  // 1/sigma^2
    float d2_series;    // leaf-pair squared gap below which the series branch may be needed
    float d2_singular;  // leaf-pair squared gap above which the singular kernel is exact
    float ks;      // sqrt(2/pi) / sigma^3 (series K prefactor)
    float fs;      // sqrt(2/pi) / sigma^5 (series F prefactor)
};

// Series of k(rho) = q/rho^3 and f(rho) = k'(rho)/rho in x = rho^2 (integrating the Gaussian
// shell density term by term: q = sqrt(2/pi) sum_k (-1)^k rho^(2k+3) / (2^k k! (2k+3))).
template <typename T> __device__ __forceinline__ T series_k(T x)
{
    return T(1.0 / 3.0) + x * (T(-1.0 / 10.0) + x * (T(1.0 / 56.0) + x * (T(-1.0 / 432.0) + x * T(1.0 / 4224.0))));
}
template <typename T> __device__ __forceinline__ T series_f(T x)
{
    return T(-1.0 / 5.0) + x * (T(1.0 / 14.0) + x * (T(-1.0 / 72.0) + x * (T(1.0 / 528.0) + x * T(-1.0 / 4992.0))));
}

struct Acc {
    float u0, u1, u2, a0, a1, a2, b0, b1, b2;
};

__device__ __forceinline__ void pair_f32(const P2PConst &k, float xi0, float xi1, float xi2, float gi0, float gi1,
                                         float gi2, float4 xj, float4 gj, Acc &acc)
{
    float dx = xi0 - xj.x, dy = xi1 - xj.y, dz = xi2 - xj.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float z = r2 * k.ce;
    float e = ex2_approx(z);
    float rinv = rsqrt_approx(r2);
    float r = r2 * rinv;
    float t = rcp_approx(fmaf(r, k.ct, 1.0f));
    float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                          0.254829592f);
    float q = fmaf(-e, fmaf(k.cq, r, poly), 1.0f);
    float rinv2 = rinv * rinv;
    float K = q * (rinv2 * rinv);
    float F = rinv2 * fmaf(-3.0f, K, k.cf * e);
    if (z > k.zs) {  // rho < 0.5 (including the self pair, r2 = 0)
        float x = r2 * k.inv_s2;
        K = k.ks * series_k<float>(x);
        F = k.fs * series_f<float>(x);
    }
    float w0 = gj.y * dz - gj.z * dy;
    float w1 = gj.z * dx - gj.x * dz;
    float w2 = gj.x * dy - gj.y * dx;
    acc.u0 = fmaf(K, w0, acc.u0);
    acc.u1 = fmaf(K, w1, acc.u1);
    acc.u2 = fmaf(K, w2, acc.u2);
    acc.a0 = fmaf(K, gj.x, acc.a0);
    acc.a1 = fmaf(K, gj.y, acc.a1);
    acc.a2 = fmaf(K, gj.z, acc.a2);
    float fg = F * fmaf(gi0, dx, fmaf(gi1, dy, gi2 * dz));
    acc.b0 = fmaf(fg, w0, acc.b0);
    acc.b1 = fmaf(fg, w1, acc.b1);
    acc.b2 = fmaf(fg, w2, acc.b2);
}

// --- FP32 near-field kernel in scaled, leaf-relative coordinates -------------------------
// Positions enter as x^ = s (x - z_t), z_t the target leaf centre, s = sqrt(log2(e)/(2 sigma^2)),
// so that exp(-rho^2/2) = 2^(-|r^|^2) needs no multiply; every other sigma factor folds into
// constants.  With c_j = gamma_j x x^_j (formed once per source when it is staged),
//   sum K gamma_j x r^ = A x x^_i - U,         A = sum K gamma_j,   U = sum K c_j,
//   sum f (gamma_j x r^) = D x x^_i - E,       D = sum f gamma_j,   E = sum f c_j,
// with f = F (gamma_i . r^), which saves the per-pair cross product.  Leaf-relative
// coordinates keep |x^_i| within a few |r^| of the nearest pairs, so the rearrangement costs
// at most a few FP32 ulps.
struct P3Const {
    float s;           // coordinate scale
    float ct;          // A&S p / (sqrt2 sigma s)
    float cq;          // sqrt(2/pi) / (sigma s)
    float cf;          // sqrt(2/pi) / (sigma^3 s^3)
    float r2s;         // |r^|^2 below which rho < 0.5
    float inv_s2;      // 1 / (sigma s)^2: rho^2 = |r^|^2 inv_s2
    float ks, fs;      // series prefactors sqrt(2/pi)/(sigma s)^3 and /(sigma s)^5
    float d2_series;   // leaf-box squared gap (true units) below which rho < 0.5 may occur
    float d2_singular; // leaf-box squared gap (true units) above which rho >= 6.5
    float d2_cut;      // (rho_cut sigma)^2: beyond the near rings, octants closer than this are corrected
    float w2_lo;       // leaf width squared, less a rounding margin
    float L;
};

// In the scaled coordinates sigma s = sqrt(log2(e) / 2) whatever sigma is, so every constant of
// the pair arithmetic is a fixed number.  The erf polynomial's coefficients are compiled in as
// immediates (2.5 % faster than reading them from the kernel parameters at 256^3);
// VFMM_P3_IMM=1 compiles the sigma-derived constants in as well (measured 0.3 % slower).
constexpr double P3_SS = 0.84932180028801904272;  // sigma s = sqrt(log2(e) / 2)
constexpr double P3_CPI = 0.79788456080286535588;  // sqrt(2 / pi)
constexpr float P3_CT = (float)(0.3275911 / (1.41421356237309504880 * P3_SS));
constexpr float P3_CQ = (float)(P3_CPI / P3_SS);
constexpr float P3_CF = (float)(P3_CPI / (P3_SS * P3_SS * P3_SS));
constexpr float P3_R2S = (float)(0.25 * P3_SS * P3_SS);
constexpr float P3_INV_S2 = (float)(1.0 / (P3_SS * P3_SS));
constexpr float P3_FS = (float)(P3_CPI / (P3_SS * P3_SS * P3_SS * P3_SS * P3_SS));

#ifndef VFMM_P3_IMM
#define VFMM_P3_IMM 0
#endif
#if VFMM_P3_IMM
#define P3K_CT P3_CT
#define P3K_CQ P3_CQ
#define P3K_CF P3_CF
#define P3K_R2S P3_R2S
#define P3K_INV_S2 P3_INV_S2
#define P3K_KS P3_CF
#define P3K_FS P3_FS
#else
#define P3K_CT k.ct
#define P3K_CQ k.cq
#define P3K_CF k.cf
#define P3K_R2S k.r2s
#define P3K_INV_S2 k.inv_s2
#define P3K_KS k.ks
#define P3K_FS k.fs
#endif

// t P(t) of A&S 7.1.26: erfc(x) = t P(t) exp(-x^2), t = 1/(1 + p x)
__device__ __forceinline__ float as_poly(const P3Const &, float t)
{
    return t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                    0.254829592f);
}

struct Acc3 {
    float A0, A1, A2, U0, U1, U2, D0, D1, D2, E0, E1, E2;
};

template <int MODE>
__device__ __forceinline__ void pair3(const P3Const &k, float xi0, float xi1, float xi2, float gi0, float gi1, float gi2,
                                      const float4 &xj, const float4 &gj, const float4 &cj, Acc3 &a)
{
    float dx = xi0 - xj.x, dy = xi1 - xj.y, dz = xi2 - xj.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float K, F;
    if (MODE == 3) {  // smoothed minus singular: the far field's missing Gaussian tail
        float e = ex2_approx(-r2);
        float rinv = rsqrt_approx(r2);
        float r = r2 * rinv;
        float t = rcp_approx(fmaf(r, P3K_CT, 1.0f));
        float poly = as_poly(k, t);
        float omq = e * fmaf(P3K_CQ, r, poly);  // 1 - q(rho)
        float rinv2 = rinv * rinv;
        K = -omq * (rinv2 * rinv);
        F = rinv2 * fmaf(-3.0f, K, P3K_CF * e);
    } else if (MODE == 2) {  // singular kernel: K = 1/r^3, F = -3/r^5
        float rinv = rsqrt_approx(r2);
        float rinv2 = rinv * rinv;
        K = rinv2 * rinv;
        F = -3.0f * K * rinv2;
    } else {
        float e = ex2_approx(-r2);
        float rinv = rsqrt_approx(r2);
        float r = r2 * rinv;
        float t = rcp_approx(fmaf(r, P3K_CT, 1.0f));
        float poly = as_poly(k, t);
        float q = fmaf(-e, fmaf(P3K_CQ, r, poly), 1.0f);
        float rinv2 = rinv * rinv;
        K = q * (rinv2 * rinv);
        F = rinv2 * fmaf(-3.0f, K, P3K_CF * e);
        if (MODE == 0) {
            if (r2 < P3K_R2S) {  // rho < 0.5, including the self pair
                float x = r2 * P3K_INV_S2;
                K = P3K_KS * series_k<float>(x);
                F = P3K_FS * series_f<float>(x);
            }
        }
    }
    a.A0 = fmaf(K, gj.x, a.A0);
    a.A1 = fmaf(K, gj.y, a.A1);
    a.A2 = fmaf(K, gj.z, a.A2);
    a.U0 = fmaf(K, cj.x, a.U0);
    a.U1 = fmaf(K, cj.y, a.U1);
    a.U2 = fmaf(K, cj.z, a.U2);
    float f = F * fmaf(gi0, dx, fmaf(gi1, dy, gi2 * dz));
    a.D0 = fmaf(f, gj.x, a.D0);
    a.D1 = fmaf(f, gj.y, a.D1);
    a.D2 = fmaf(f, gj.z, a.D2);
    a.E0 = fmaf(f, cj.x, a.E0);
    a.E1 = fmaf(f, cj.y, a.E1);
    a.E2 = fmaf(f, cj.z, a.E2);
}

// Tuning knobs (compile-time): targets per lane, the unroll of the source loop, blocks per SM.
// In-line P2P at 256^3 (sigma = h), before the full-tile loop: two targets per lane, unroll 1,
// 32 blocks per SM 50.2 ms; unroll 2 50.4; 28 blocks per SM 50.9; 16 blocks per SM (128
// registers) 54.7; four targets per lane with the half-warp split (VFMM_P3_SPLIT) 52.5 at 16
// and 56.8 at 20 blocks per SM.  After the warp-parallel octant classification (44.5 ms at
// 32 blocks per SM), the full-tile loop unrolled 2 / 4 / 8 / 16 / 32: 44.7 / 44.4 / 43.6 /
// 45.8 / 58.4 ms; unroll 8 at 28 / 24 blocks per SM: 43.4 / 44.2 ms.
#ifndef VFMM_P3_TPT
#define VFMM_P3_TPT 2
#endif
#ifndef VFMM_P3_UNROLL
#define VFMM_P3_UNROLL 1
#endif
// VFMM_P3_SPLIT = 1: four targets per lane, the two half-warps taking alternate sources of every
// run (their sums are added by one shuffle at the end), which halves the per-source overhead
// (loads, loop, uniform-datapath and move instructions) per pair.
#ifndef VFMM_P3_SPLIT
#define VFMM_P3_SPLIT 0
#endif
constexpr int P3_SPLIT = VFMM_P3_SPLIT;
// VFMM_P3_HALF_CULL = 1: the ring-2 correction is culled per (half of the warp's targets, source
// octant) instead of per (target leaf, source octant).  The two targets of a lane are q = 0 (the
// first 32 of the chunk) and q = 1 (the next 32); the leaf's particles are sorted by octant, so
// on a regular distribution the halves are the leaf's two x-halves.
#ifndef VFMM_P3_HALF_CULL
#define VFMM_P3_HALF_CULL 1
#endif
constexpr int P3_THREADS = 32;                            // one warp per target leaf chunk
constexpr int P3_TPT = P3_SPLIT ? 4 : VFMM_P3_TPT;        // targets per lane
constexpr int P3_LANES = P3_SPLIT ? 16 : 32;              // lanes that share one source
constexpr bool P3_HALVES = VFMM_P3_HALF_CULL && !P3_SPLIT && P3_TPT == 2;
constexpr int P3_TARGETS = P3_LANES * P3_TPT;             // targets per block
constexpr int P3_TILE = 64;      // staged sources
constexpr int P3_UNROLL = VFMM_P3_UNROLL;

// one staged source: scaled position relative to the target leaf centre, strength, and
// c = gamma x x (the cross product the velocity sum needs, formed once per source)
struct __align__(16) Src3 {
    float4 x, g, c;
};

template <int MODE>
__device__ __forceinline__ void tile3(const P3Const &k, const float (&xi)[P3_TPT][3], const float (&gi)[P3_TPT][3],
                                      const Src3 *src, int j0, int j1, Acc3 (&acc)[P3_TPT])
{
#pragma unroll P3_UNROLL
    for (int j = j0; j < j1; j += 1 + P3_SPLIT) {
        const float4 xj = src[j].x, gj = src[j].g, cj = src[j].c;
#pragma unroll
        for (int q = 0; q < P3_TPT; ++q) pair3<MODE>(k, xi[q][0], xi[q][1], xi[q][2], gi[q][0], gi[q][1], gi[q][2], xj, gj, cj, acc[q]);
    }
}

// The general loop for the targets of one half only (QM = 1: q = 0, QM = 2: q = 1): a ring-2
// octant that only one half of the warp's targets comes within rho_cut sigma of.
template <int MODE, int QM>
__device__ __forceinline__ void tile3q(const P3Const &k, const float (&xi)[P3_TPT][3], const float (&gi)[P3_TPT][3],
                                       const Src3 *src, int j0, int j1, Acc3 (&acc)[P3_TPT])
{
#pragma unroll P3_UNROLL
    for (int j = j0; j < j1; ++j) {
        const float4 xj = src[j].x, gj = src[j].g, cj = src[j].c;
#pragma unroll
        for (int q = 0; q < P3_TPT; ++q)
            if ((QM >> q) & 1)
                pair3<MODE>(k, xi[q][0], xi[q][1], xi[q][2], gi[q][0], gi[q][1], gi[q][2], xj, gj, cj, acc[q]);
    }
}

// A whole staged tile with one inner loop (the common case: every octant of a near-ring leaf
// takes the same kernel): a compile-time trip count lets the loads use immediate offsets and
// drops most of the per-source loop control.
#ifndef VFMM_P3_FULLTILE
#define VFMM_P3_FULLTILE 8  // unroll of the full-tile loop; 0 = the general loop only
#endif
constexpr int P3_FULL_UNROLL = VFMM_P3_FULLTILE > 0 ? VFMM_P3_FULLTILE : 1;
template <int MODE>
__device__ __forceinline__ void tile3_full(const P3Const &k, const float (&xi)[P3_TPT][3], const float (&gi)[P3_TPT][3],
                                           const Src3 *src, Acc3 (&acc)[P3_TPT])
{
#pragma unroll P3_FULL_UNROLL
    for (int j = 0; j < P3_TILE; ++j) {
        const float4 xj = src[j].x, gj = src[j].g, cj = src[j].c;
#pragma unroll
        for (int q = 0; q < P3_TPT; ++q) pair3<MODE>(k, xi[q][0], xi[q][1], xi[q][2], gi[q][0], gi[q][1], gi[q][2], xj, gj, cj, acc[q]);
    }
}

struct AccD {
    double u0, u1, u2, a0, a1, a2, b0, b1, b2;
};

// FP64 pair: q from erf/exp of the CUDA math library, series below rho = 0.5.
__device__ __forceinline__ void pair_f64(double sigma, double xi0, double xi1, double xi2, double gi0, double gi1,
                                         double gi2, dvec4 xj, dvec4 gj, AccD &acc)
{
    const double c = 0.79788456080286535588;  // sqrt(2/pi)
    double dx = xi0 - xj.x, dy = xi1 - xj.y, dz = xi2 - xj.z;
    double r2 = dx * dx + dy * dy + dz * dz;
    double s2 = sigma * sigma;
    double x = r2 / s2;
    double K, F;
    if (x < 0.25) {
        // the same two series summed to FP64 convergence
        double kk = 0.0, ff = 0.0, xp = 1.0, xm1 = 1.0, fact = 1.0;  // xp = x^q, xm1 = x^(q-1), fact = 2^q q!
        for (int q = 0; q < 16; ++q) {
            double den = fact * (2 * q + 3);
            kk += (q & 1) ? -xp / den : xp / den;
            if (q >= 1) ff += (q & 1) ? -2.0 * q * xm1 / den : 2.0 * q * xm1 / den;
            xm1 = xp;
            xp *= x;
            fact *= 2.0 * (q + 1);
        }
        K = c / (s2 * sigma) * kk;
        F = c / (s2 * s2 * sigma) * ff;
    } else {
        double r = sqrt(r2);
        double rho = r / sigma;
        double e = exp(-0.5 * x);
        double q = erf(rho * 0.70710678118654752440) - c * rho * e;
        K = q / (r2 * r);
        F = (c * e / (s2 * sigma) - 3.0 * K) / r2;
    }
    double w0 = gj.y * dz - gj.z * dy;
    double w1 = gj.z * dx - gj.x * dz;
    double w2 = gj.x * dy - gj.y * dx;
    acc.u0 += K * w0;
    acc.u1 += K * w1;
    acc.u2 += K * w2;
    acc.a0 += K * gj.x;
    acc.a1 += K * gj.y;
    acc.a2 += K * gj.z;
    double fg = F * (gi0 * dx + gi1 * dy + gi2 * dz);
    acc.b0 += fg * w0;
    acc.b1 += fg * w1;
    acc.b2 += fg * w2;
}

template <typename TOut>
__device__ __forceinline__ void store_out(TOut *u_out, TOut *s_out, int i, double u0, double u1, double u2,
                                          double s0, double s1, double s2)
{
    u_out[3 * (int64_t)i + 0] = (TOut)u0;
    u_out[3 * (int64_t)i + 1] = (TOut)u1;
    u_out[3 * (int64_t)i + 2] = (TOut)u2;
    if (s_out) {
        s_out[3 * (int64_t)i + 0] = (TOut)s0;
        s_out[3 * (int64_t)i + 1] = (TOut)s1;
        s_out[3 * (int64_t)i + 2] = (TOut)s2;
    }
}

constexpr int P2P_BS = 64;
constexpr float INV_4PI_F = 0.0795774715459476679f;
constexpr double INV_4PI_D = 0.0795774715459476679;

#if VFMM_CHECK
// checked build: source-target pairs the FP32 P2P computed for real targets (the accounting
// behind the benchmark's roofline, compared with its host-side count by a test)
__device__ unsigned long long g_p2p_pairs;
#endif

#ifndef VFMM_P3_MINB
#if VFMM_P3_SPLIT
#define VFMM_P3_MINB 20  // 20 one-warp blocks per SM (102 registers: four targets per lane)
#else
#define VFMM_P3_MINB 28  // 28 one-warp blocks per SM (73 registers)
#endif
#endif
#if VFMM_P3_MINB > 0
#define VFMM_P3_BOUNDS __launch_bounds__(P3_THREADS, VFMM_P3_MINB)
#else
#define VFMM_P3_BOUNDS __launch_bounds__(P3_THREADS)
#endif
__global__ void VFMM_P3_BOUNDS k_p2p_f32(const float4 *__restrict__ xs, const float4 *__restrict__ gs,
                                                        const int *__restrict__ ls, const float4 *__restrict__ bbox,
                                                        const int *__restrict__ oct_start,
                                                        const float4 *__restrict__ oct_box, int nside, int log2n,
                                                        int R, int Rc, int direct_K, float leaf_w, P3Const kc,
                                                        const float *__restrict__ ufar, const float *__restrict__ sfar,
                                                        const int *__restrict__ perm, float *__restrict__ u_out,
                                                        float *__restrict__ s_out, int *__restrict__ err, int chunks,
                                                        int64_t ntask)
{
    __shared__ Src3 src[P3_TILE];
    __shared__ int ost[9];
    __shared__ float hbox[2][6];  // boxes (true units) of the two target halves: lo xyz, hi xyz
    const float s = kc.s;
    // tasks = (leaf, chunk of P3_TARGETS targets); the grid is either one block per task or a
    // persistent grid that strides over them
    for (int64_t task = blockIdx.x; task < ntask; task += gridDim.x) {
    const int leaf = (int)(task / chunks), chunk = (int)(task - (int64_t)leaf * chunks);
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const int tb = ls[leaf], te = ls[leaf + 1];
    const float zx = (cx + 0.5f) * leaf_w, zy = (cy + 0.5f) * leaf_w, zz = (cz + 0.5f) * leaf_w;
    const float4 tlo = bbox[2 * leaf], thi = bbox[2 * leaf + 1];
    for (int t0 = tb + chunk * P3_TARGETS; t0 < te; t0 += chunks * P3_TARGETS) {
        float xi[P3_TPT][3], gi[P3_TPT][3];
        int tix[P3_TPT];
#pragma unroll
        for (int q = 0; q < P3_TPT; ++q) {
            int ti = t0 + (int)(threadIdx.x % P3_LANES) + q * P3_LANES;
            tix[q] = ti;
            float4 x = ti < te ? xs[ti] : make_float4(zx, zy, zz, 0.f);
            float4 g = ti < te ? gs[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
            xi[q][0] = s * (x.x - zx);
            xi[q][1] = s * (x.y - zy);
            xi[q][2] = s * (x.z - zz);
            gi[q][0] = g.x;
            gi[q][1] = g.y;
            gi[q][2] = g.z;
            if (P3_HALVES) {
                // box of this half's targets (empty halves give lo > hi, so no octant is near)
                const bool act = ti < te;
                float b[6] = {act ? x.x : 3e38f, act ? x.y : 3e38f, act ? x.z : 3e38f,
                              act ? x.x : -3e38f, act ? x.y : -3e38f, act ? x.z : -3e38f};
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        b[d] = fminf(b[d], __shfl_xor_sync(0xffffffffu, b[d], off));
                        b[3 + d] = fmaxf(b[3 + d], __shfl_xor_sync(0xffffffffu, b[3 + d], off));
                    }
                __syncwarp();
                if ((threadIdx.x & 31) == 0)
#pragma unroll
                    for (int d = 0; d < 6; ++d) hbox[q & 1][d] = b[d];
            }
        }
        if (P3_HALVES) __syncwarp();
        Acc3 acc[P3_TPT];
#pragma unroll
        for (int q = 0; q < P3_TPT; ++q) acc[q] = Acc3{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        // neighbour offsets: the (2R+1)^3 near field, or for the direct sum every leaf of the
        // (2K+1)^3 image boxes
        int lo[3], hi[3];
        const int cc[3] = {cx, cy, cz};
        // the near rings R (full smoothed kernel) and, out to Rc, the correction rings; for the
        // direct sum every leaf of the (2K+1)^3 image boxes
        const int Rl = direct_K >= 0 ? 0 : (Rc > R ? Rc : R);
        for (int d = 0; d < 3; ++d) {
            lo[d] = direct_K >= 0 ? -cc[d] - direct_K * nside : -Rl;
            hi[d] = direct_K >= 0 ? nside - 1 - cc[d] + direct_K * nside : Rl;
        }
        // Neighbour leaves in batches of four: lane (li, o) classifies octant o of neighbour li
        // of the batch by the closest approach of the target leaf box and the octant box (in the
        // near rings smoothed with or without the small-rho series, or singular; beyond them the
        // Gaussian-tail correction for octants closer than rho_cut sigma (mode 3), nothing
        // otherwise (mode 4, the M2L has them)); three ballots give every lane the modes of all
        // 32 octants, so the warp-uniform loop below reads its inner-loop choice per octant.  A
        // mode-3 octant is then tested against the box of each half of the warp's targets (q = 0,
        // 1), and two more ballots say which halves its pairs run for.
        const int n1 = hi[1] - lo[1] + 1, n2 = hi[2] - lo[2] + 1;
        const int n_off = (hi[0] - lo[0] + 1) * n1 * n2;
        const int lane = threadIdx.x & 31;
        for (int idx0 = 0; idx0 < n_off; idx0 += 4) {
            int my_mode = 4, my_q = 3;  // my_q: the target halves an octant of mode 3 is near
            {
                const int idx = idx0 + (lane >> 3), o = lane & 7;
                if (idx < n_off) {
                    const int ox = lo[0] + idx / (n1 * n2), oy = lo[1] + (idx / n2) % n1, oz = lo[2] + idx % n2;
                    const bool corr = direct_K < 0 && (abs(ox) > R || abs(oy) > R || abs(oz) > R);
                    // the cells alone keep a leaf |o| rings away at least (|o| - 1) w apart along
                    // that axis: a correction-ring leaf that cannot come within rho_cut sigma is skipped
                    const float cgx = (float)max(abs(ox) - 1, 0), cgy = (float)max(abs(oy) - 1, 0),
                                cgz = (float)max(abs(oz) - 1, 0);
                    if (!corr || (cgx * cgx + cgy * cgy + cgz * cgz) * kc.w2_lo < kc.d2_cut) {
                        const int nx = cx + ox, ny = cy + oy, nz = cz + oz;
                        int sl = ((nx & (nside - 1)) * nside + (ny & (nside - 1))) * nside + (nz & (nside - 1));
                        sl = checked_index(sl, nside * nside * nside, err);
                        const float shx = kc.L * (float)(nx >> log2n), shy = kc.L * (float)(ny >> log2n),
                                    shz = kc.L * (float)(nz >> log2n);
                        const float4 slo = oct_box[16 * sl + 2 * o], shi = oct_box[16 * sl + 2 * o + 1];
                        const float gx = fmaxf(0.f, fmaxf(slo.x + shx - thi.x, tlo.x - shi.x - shx));
                        const float gy = fmaxf(0.f, fmaxf(slo.y + shy - thi.y, tlo.y - shi.y - shy));
                        const float gz = fmaxf(0.f, fmaxf(slo.z + shz - thi.z, tlo.z - shi.z - shz));
                        const float d2 = gx * gx + gy * gy + gz * gz;
                        my_mode = corr ? (d2 < kc.d2_cut ? 3 : 4)
                                       : (d2 >= kc.d2_singular ? 2 : (d2 >= kc.d2_series ? 1 : 0));
                        if (P3_HALVES && my_mode == 3) {
                            my_q = 0;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const float hx = fmaxf(0.f, fmaxf(slo.x + shx - hbox[h][3], hbox[h][0] - shi.x - shx));
                                const float hy = fmaxf(0.f, fmaxf(slo.y + shy - hbox[h][4], hbox[h][1] - shi.y - shy));
                                const float hz = fmaxf(0.f, fmaxf(slo.z + shz - hbox[h][5], hbox[h][2] - shi.z - shz));
                                if (hx * hx + hy * hy + hz * hz < kc.d2_cut) my_q |= 1 << h;
                            }
                            if (my_q == 0) my_mode = 4;
                        }
                    }
                }
            }
            const unsigned b0 = __ballot_sync(0xffffffffu, my_mode & 1), b1 = __ballot_sync(0xffffffffu, my_mode & 2),
                           b2 = __ballot_sync(0xffffffffu, my_mode & 4);
            // halves of the warp's targets that a mode-3 octant is near (both for every other mode)
            const unsigned bh0 = P3_HALVES ? __ballot_sync(0xffffffffu, my_q & 1) : 0xffffffffu,
                           bh1 = P3_HALVES ? __ballot_sync(0xffffffffu, my_q & 2) : 0xffffffffu;
            for (int li = 0; li < 4; ++li) {
                const int idx = idx0 + li;
                if (idx >= n_off) break;
                const unsigned m0 = (b0 >> (8 * li)) & 0xFFu, m1 = (b1 >> (8 * li)) & 0xFFu,
                               m2 = (b2 >> (8 * li)) & 0xFFu, h0 = (bh0 >> (8 * li)) & 0xFFu,
                               h1 = (bh1 >> (8 * li)) & 0xFFu;
                if (m2 == 0xFFu && (m0 | m1) == 0u) continue;  // all eight octants: nothing to add
                const int ox = lo[0] + idx / (n1 * n2), oy = lo[1] + (idx / n2) % n1, oz = lo[2] + idx % n2;
                const int nx = cx + ox, ny = cy + oy, nz = cz + oz;
                int sl = ((nx & (nside - 1)) * nside + (ny & (nside - 1))) * nside + (nz & (nside - 1));
                sl = checked_index(sl, nside * nside * nside, err);
                const float shx = kc.L * (float)(nx >> log2n), shy = kc.L * (float)(ny >> log2n),
                            shz = kc.L * (float)(nz >> log2n);
                // sources relative to the target leaf centre, with the image shift
                const float ox0 = shx - zx, ox1 = shy - zy, ox2 = shz - zz;
                const int sb = ls[sl], se = ls[sl + 1];
                __syncwarp();
                if (threadIdx.x < 8) ost[threadIdx.x] = oct_start[8 * sl + threadIdx.x];
                if (threadIdx.x == 8) ost[8] = se - sb;
                for (int s0 = sb; s0 < se; s0 += P3_TILE) {
                    const int cnt = min(P3_TILE, se - s0);
                    __syncwarp();
                    for (int j = threadIdx.x; j < cnt; j += P3_THREADS) {
                        float4 x = xs[s0 + j], g = gs[s0 + j];
                        float a0 = s * (x.x + ox0), a1 = s * (x.y + ox1), a2 = s * (x.z + ox2);
                        src[j].x = make_float4(a0, a1, a2, 0.f);
                        src[j].g = g;
                        src[j].c = make_float4(g.y * a2 - g.z * a1, g.z * a0 - g.x * a2, g.x * a1 - g.y * a0, 0.f);
                    }
                    __syncwarp();
                    const int c0 = s0 - sb, c1 = c0 + cnt;
                    // runs of consecutive octants with the same inner loop (mode, and for mode 3
                    // the target halves it serves)
                    auto run_key = [&](int oo) {
                        return (int)(((m0 >> oo) & 1u) | (((m1 >> oo) & 1u) << 1) | (((m2 >> oo) & 1u) << 2) |
                                     (((h0 >> oo) & 1u) << 3) | (((h1 >> oo) & 1u) << 4));
                    };
                    int o = 0;
                    while (o < 8) {
                        const int key = run_key(o);
                        const int mode = key & 7, qm = key >> 3;
                        int o2 = o + 1;
                        while (o2 < 8 && run_key(o2) == key) ++o2;
                        const int j0 = max(ost[o], c0) - c0, j1 = min(ost[o2], c1) - c0;
#if VFMM_CHECK
                        if (!P3_SPLIT && mode < 4 && j0 < j1 && (threadIdx.x & 31) == 0) {
                            // targets of this chunk in each half that the run serves
                            const int na0 = min(max(te - t0, 0), P3_LANES), na1 = min(max(te - t0 - P3_LANES, 0), P3_LANES);
                            const int qmr = mode == 3 ? qm : 3;
                            const int nt = ((qmr & 1) ? na0 : 0) + ((qmr & 2) ? na1 : 0);
                            atomicAdd(&g_p2p_pairs, (unsigned long long)(j1 - j0) * (unsigned long long)nt);
                        }
#endif
                        if (mode == 3 && qm != 3) {
                            if (j0 < j1) {
                                if (qm == 1) tile3q<3, 1>(kc, xi, gi, src, j0, j1, acc);
                                else tile3q<3, 2>(kc, xi, gi, src, j0, j1, acc);
                            }
                        } else if (VFMM_P3_FULLTILE > 0 && !P3_SPLIT && j0 == 0 && j1 == P3_TILE && (mode == 1 || mode == 3)) {
                            if (mode == 1) tile3_full<1>(kc, xi, gi, src, acc);
                            else tile3_full<3>(kc, xi, gi, src, acc);
                        } else if (j0 < j1) {
                            const int jh = j0 + (P3_SPLIT ? (int)(threadIdx.x >> 4) : 0);
                            if (mode == 2) tile3<2>(kc, xi, gi, src, jh, j1, acc);
                            else if (mode == 1) tile3<1>(kc, xi, gi, src, jh, j1, acc);
                            else if (mode == 0) tile3<0>(kc, xi, gi, src, jh, j1, acc);
                            else if (mode == 3) tile3<3>(kc, xi, gi, src, jh, j1, acc);
                        }
                        o = o2;
                    }
                }
            }
        }
        if (P3_SPLIT) {
            // the two half-warps summed alternate sources: add them
#pragma unroll
            for (int q = 0; q < P3_TPT; ++q) {
                float *v = &acc[q].A0;
#pragma unroll
                for (int e = 0; e < 12; ++e) v[e] += __shfl_xor_sync(0xffffffffu, v[e], 16);
            }
        }
        // u = s^2 (A x x^ - U), S = s^3 (A x gamma + D x x^ - E), times 1/(4 pi)
        const float su = INV_4PI_F * s * s, ss = su * s;
#pragma unroll
        for (int q = 0; q < P3_TPT; ++q) {
            int ti = tix[q];
            if (P3_SPLIT && (q >> 1) != (int)(threadIdx.x >> 4)) continue;  // each half writes two targets
            if (ti >= te) continue;
            const Acc3 &a = acc[q];
            const float *x = xi[q], *g = gi[q];
            float u0 = su * (a.A1 * x[2] - a.A2 * x[1] - a.U0);
            float u1 = su * (a.A2 * x[0] - a.A0 * x[2] - a.U1);
            float u2 = su * (a.A0 * x[1] - a.A1 * x[0] - a.U2);
            float s0 = ss * (a.A1 * g[2] - a.A2 * g[1] + a.D1 * x[2] - a.D2 * x[1] - a.E0);
            float s1 = ss * (a.A2 * g[0] - a.A0 * g[2] + a.D2 * x[0] - a.D0 * x[2] - a.E1);
            float s2 = ss * (a.A0 * g[1] - a.A1 * g[0] + a.D0 * x[1] - a.D1 * x[0] - a.E2);
            if (ufar) {
                u0 += ufar[3 * (int64_t)ti + 0];
                u1 += ufar[3 * (int64_t)ti + 1];
                u2 += ufar[3 * (int64_t)ti + 2];
                s0 += sfar[3 * (int64_t)ti + 0];
                s1 += sfar[3 * (int64_t)ti + 1];
                s2 += sfar[3 * (int64_t)ti + 2];
            }
            store_out<float>(u_out, s_out, perm[ti], u0, u1, u2, s0, s1, s2);
        }
    }
    }  // task
}

__global__ void __launch_bounds__(P2P_BS) k_p2p_f64(const dvec4 *__restrict__ xs, const dvec4 *__restrict__ gs,
                                                    const int *__restrict__ ls, int nside, int log2n, int R,
                                                    int direct_K, double sigma, double L,
                                                    const double *__restrict__ ufar,
                                                    const double *__restrict__ sfar, const int *__restrict__ perm,
                                                    double *__restrict__ u_out, double *__restrict__ s_out)
{
    __shared__ dvec4 sx[P2P_BS];
    __shared__ dvec4 sg[P2P_BS];
    const int leaf = blockIdx.x;
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const int tb = ls[leaf], te = ls[leaf + 1];
    for (int t0 = tb + blockIdx.y * P2P_BS; t0 < te; t0 += gridDim.y * P2P_BS) {
        const int ti = t0 + threadIdx.x;
        const bool active = ti < te;
        dvec4 z4 = {0, 0, 0, 0};
        dvec4 xi = active ? xs[ti] : z4;
        dvec4 gi = active ? gs[ti] : z4;
        AccD acc = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        int lo[3], hi[3];
        const int cc[3] = {cx, cy, cz};
        for (int d = 0; d < 3; ++d) {
            lo[d] = direct_K >= 0 ? -cc[d] - direct_K * nside : -R;
            hi[d] = direct_K >= 0 ? nside - 1 - cc[d] + direct_K * nside : R;
        }
        for (int ox = lo[0]; ox <= hi[0]; ++ox)
            for (int oy = lo[1]; oy <= hi[1]; ++oy)
                for (int oz = lo[2]; oz <= hi[2]; ++oz) {
                    int nx = cx + ox, ny = cy + oy, nz = cz + oz;
                    int sl = ((nx & (nside - 1)) * nside + (ny & (nside - 1))) * nside + (nz & (nside - 1));
                    double xi0 = xi.x - L * (double)(nx >> log2n);
                    double xi1 = xi.y - L * (double)(ny >> log2n);
                    double xi2 = xi.z - L * (double)(nz >> log2n);
                    int sb = ls[sl], se = ls[sl + 1];
                    for (int s0 = sb; s0 < se; s0 += P2P_BS) {
                        int cnt = min(P2P_BS, se - s0);
                        __syncthreads();
                        if (threadIdx.x < cnt) {
                            sx[threadIdx.x] = xs[s0 + threadIdx.x];
                            sg[threadIdx.x] = gs[s0 + threadIdx.x];
                        }
                        __syncthreads();
                        for (int j = 0; j < cnt; ++j) pair_f64(sigma, xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j], sg[j], acc);
                    }
                }
        if (active) {
            double s0 = acc.a1 * gi.z - acc.a2 * gi.y + acc.b0;
            double s1 = acc.a2 * gi.x - acc.a0 * gi.z + acc.b1;
            double s2 = acc.a0 * gi.y - acc.a1 * gi.x + acc.b2;
            double u0 = acc.u0 * INV_4PI_D, u1 = acc.u1 * INV_4PI_D, u2 = acc.u2 * INV_4PI_D;
            s0 *= INV_4PI_D;
            s1 *= INV_4PI_D;
            s2 *= INV_4PI_D;
            if (ufar) {
                u0 += ufar[3 * (int64_t)ti + 0];
                u1 += ufar[3 * (int64_t)ti + 1];
                u2 += ufar[3 * (int64_t)ti + 2];
                s0 += sfar[3 * (int64_t)ti + 0];
                s1 += sfar[3 * (int64_t)ti + 1];
                s2 += sfar[3 * (int64_t)ti + 2];
            }
            store_out<double>(u_out, s_out, perm[ti], u0, u1, u2, s0, s1, s2);
        }
    }
}

void set_carveouts_p2p() { prefer_max_shared(k_p2p_f32); }

// Pair counter of the checked build (0 in the default build): reset before a launch, read after.
int64_t p2p_pairs_read()
{
#if VFMM_CHECK
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_p2p_pairs, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int64_t)v;
#else
    return 0;
#endif
}

int launch_p2p(Ctx *c, int R, int Rc, double sigma, const void *ufar, const void *sfar, void *u_out, void *s_out,
               int direct_K)
{
#if VFMM_CHECK
    {
        const unsigned long long zero = 0;
        cudaMemcpyToSymbolAsync(g_p2p_pairs, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, c->stream);
    }
#endif
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    int chunks = (c->max_leaf + P2P_BS - 1) / P2P_BS;
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    dim3 grid((unsigned)c->nleaf, (unsigned)chunks);
    if (c->f64) {
        k_p2p_f64<<<grid, P2P_BS, 0, c->stream>>>((const dvec4 *)c->xs.p, (const dvec4 *)c->gs.p,
                                                  (const int *)c->leaf_start.p, c->nside, log2n, R, direct_K,
                                                  sigma, c->cfg.box, (const double *)ufar, (const double *)sfar,
                                                  (const int *)c->perm.p, (double *)u_out, (double *)s_out);
    } else {
        const double log2e = 1.4426950408889634074;
        const double cpi = 0.79788456080286535588;
        const double sc = std::sqrt(log2e / (2.0 * sigma * sigma));
        const double ss = sigma * sc;
        P3Const kc;
        kc.s = (float)sc;
        kc.ct = (float)(0.3275911 / (1.41421356237309504880 * ss));
        kc.cq = (float)(cpi / ss);
        kc.cf = (float)(cpi / (ss * ss * ss));
        kc.r2s = (float)(0.25 * ss * ss);
        kc.inv_s2 = (float)(1.0 / (ss * ss));
        kc.ks = (float)(cpi / (ss * ss * ss));
        kc.fs = (float)(cpi / (ss * ss * ss * ss * ss));
        kc.d2_series = (float)(0.36 * sigma * sigma);      // (0.6 sigma)^2: margin over rho = 0.5
        kc.d2_singular = (float)(42.25 * sigma * sigma);   // (6.5 sigma)^2
        kc.d2_cut = (float)(c->cfg.rho_cut * c->cfg.rho_cut * sigma * sigma);
        kc.w2_lo = (float)(c->leaf_w * c->leaf_w * (1.0 - 1e-4));
        kc.L = (float)c->cfg.box;
        int chunks3 = (c->max_leaf + P3_TARGETS - 1) / P3_TARGETS;
        if (chunks3 < 1) chunks3 = 1;
        const int64_t ntask = c->nleaf * chunks3;
        // beside the concurrent far field the P2P runs as a persistent grid of P2P_SHARED_BLOCKS
        // one-warp blocks per SM, which leaves each SM the registers and shared memory of one
        // tensor-core M2L CTA (and of the smaller far-field kernels); alone, one block per task
        int64_t nblk = ntask;
        if (c->p2p_shared_blocks > 0) nblk = std::min<int64_t>(ntask, (int64_t)c->sm_count * c->p2p_shared_blocks);
        k_p2p_f32<<<(unsigned)nblk, P3_THREADS, 0, c->stream>>>((const float4 *)c->xs.p, (const float4 *)c->gs.p,
                                                       (const int *)c->leaf_start.p, (const float4 *)c->bbox.p,
                                                       (const int *)c->oct_start.p, (const float4 *)c->oct_box.p,
                                                       c->nside, log2n, R, Rc, direct_K, (float)c->leaf_w, kc,
                                                       (const float *)ufar, (const float *)sfar, (const int *)c->perm.p,
                                                       (float *)u_out, (float *)s_out, (int *)c->err.p, chunks3, ntask);
    }
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

}  // namespace vfmm

// ---------------------------------------------------------------------------------------
// Allocation-free direct sum.
//
// Some callers cannot allocate device memory when they call in: a host program that hands
// every byte of device memory to its own pool up front, or a latency-critical loop that must
// not pay cudaMalloc's implicit device synchronisation.  vfmm_direct_eval_noalloc serves them:
// it evaluates the same direct sum as VFMM_METHOD_DIRECT (FP32), with its only scratch (the
// wrapped positions and the strengths, packed as float4) in the file-scope array below,
// which every device that loads this library holds until the process exits.
// The paper has no counterpart of this entry point.
namespace vfmm {

constexpr int NOALLOC_MAX_N = VFMM_NOALLOC_MAX_N;
static __device__ __align__(256) float4 g_noalloc_scratch[2 * NOALLOC_MAX_N];  // 2 MiB

__global__ void k_noalloc_pack(int n, const float *__restrict__ x, const float *__restrict__ g, float L,
                               float4 *__restrict__ scratch)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float invL = 1.0f / L;
    scratch[i] = make_float4(wrap_coord<float>(x[3 * i], L, invL), wrap_coord<float>(x[3 * i + 1], L, invL),
                             wrap_coord<float>(x[3 * i + 2], L, invL), 0.f);
    scratch[NOALLOC_MAX_N + i] = make_float4(g[3 * i], g[3 * i + 1], g[3 * i + 2], 0.f);
}

__global__ void __launch_bounds__(P2P_BS) k_noalloc_direct(int n, int K, P2PConst kc,
                                                           const float4 *__restrict__ scratch,
                                                           float *__restrict__ u_out, float *__restrict__ s_out)
{
    __shared__ float4 sx[P2P_BS];
    __shared__ float4 sg[P2P_BS];
    const float4 *xs = scratch, *gs = scratch + NOALLOC_MAX_N;
    const int ti = blockIdx.x * P2P_BS + threadIdx.x;
    const bool active = ti < n;
    float4 xi = active ? xs[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 gi = active ? gs[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float Lf = (float)kc.L;
    Acc acc = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int ox = -K; ox <= K; ++ox)
        for (int oy = -K; oy <= K; ++oy)
            for (int oz = -K; oz <= K; ++oz) {
                float xi0 = xi.x - Lf * (float)ox, xi1 = xi.y - Lf * (float)oy, xi2 = xi.z - Lf * (float)oz;
                for (int s0 = 0; s0 < n; s0 += P2P_BS) {
                    int cnt = min(P2P_BS, n - s0);
                    __syncthreads();
                    if (threadIdx.x < cnt) {
                        sx[threadIdx.x] = xs[s0 + threadIdx.x];
                        sg[threadIdx.x] = gs[s0 + threadIdx.x];
                    }
                    __syncthreads();
                    for (int j = 0; j < cnt; ++j) pair_f32(kc, xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j], sg[j], acc);
                }
            }
    if (!active) return;
    float s0 = fmaf(acc.a1, gi.z, fmaf(-acc.a2, gi.y, acc.b0));
    float s1 = fmaf(acc.a2, gi.x, fmaf(-acc.a0, gi.z, acc.b1));
    float s2 = fmaf(acc.a0, gi.y, fmaf(-acc.a1, gi.x, acc.b2));
    u_out[3 * ti + 0] = acc.u0 * INV_4PI_F;
    u_out[3 * ti + 1] = acc.u1 * INV_4PI_F;
    u_out[3 * ti + 2] = acc.u2 * INV_4PI_F;
    if (s_out) {
        s_out[3 * ti + 0] = s0 * INV_4PI_F;
        s_out[3 * ti + 1] = s1 * INV_4PI_F;
        s_out[3 * ti + 2] = s2 * INV_4PI_F;
    }
}

}  // namespace vfmm

#include <mutex>

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
float4 *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

extern "C" int vfmm_direct_eval_noalloc(int64_t n, const float *x, const float *gamma, double sigma, double box,
                                        int images, float *u_out, float *s_out, void *stream)
{
    using namespace vfmm;
    if (n <= 0 || !x || !gamma || !u_out) return VFMM_ERR_ARG;
    if (n > NOALLOC_MAX_N) return VFMM_ERR_UNSUPPORTED;
    if (!(sigma > 0.0) || sigma != sigma || sigma > 1e300) return VFMM_ERR_ARG;
    if (!(box > 0.0) || box > 1e300) return VFMM_ERR_ARG;
    if (images < 0 || images > 20) return VFMM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return VFMM_ERR_CUDA;
    }
    float4 *scratch = nullptr;
    {
        // the host-side symbol is only a stand-in: look up the array's device address with the
        // device current.  Outside stream capture every call looks it up again (a host-side
        // table lookup that allocates nothing), so the address follows a module reload after
        // cudaDeviceReset; during capture the address of the last call outside capture is used.
        cudaStream_t st = (cudaStream_t)stream;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
            cudaGetLastError();
            return VFMM_ERR_CUDA;
        }
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return VFMM_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (float4 *)p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    P2PConst kc;
    kc.sigma = sigma;
    kc.L = box;
    const double log2e = 1.4426950408889634074;
    const double cpi = 0.79788456080286535588;
    kc.ce = (float)(-log2e / (2.0 * sigma * sigma));
    kc.ct = (float)(0.3275911 / (1.41421356237309504880 * sigma));
    kc.cq = (float)(cpi / sigma);
    kc.cf = (float)(cpi / (sigma * sigma * sigma));
    kc.zs = (float)(-0.25 * log2e / 2.0);
    kc.inv_s2 = (float)(1.0 / (sigma * sigma));
    kc.ks = (float)(cpi / (sigma * sigma * sigma));
    kc.fs = (float)(cpi / (sigma * sigma * sigma * sigma * sigma));
    cudaStream_t st = (cudaStream_t)stream;
    int nn = (int)n;
    k_noalloc_pack<<<(nn + 255) / 256, 256, 0, st>>>(nn, x, gamma, (float)box, scratch);
    k_noalloc_direct<<<(nn + P2P_BS - 1) / P2P_BS, P2P_BS, 0, st>>>(nn, images, kc, scratch, u_out, s_out);
    if (cudaGetLastError() != cudaSuccess) return VFMM_ERR_CUDA;
    return VFMM_OK;
}

// ---------------------------------------------------------------------------------------
// Velocity gradient at the particles (near field), for the adjoint:
//   du_a/dx_k = sum_j [ K eps_abk gamma_jb + F (gamma_j x r)_a r_k ]
// (the derivative of K(r) gamma_j x r; the oracle writes the same sum).
namespace vfmm {

template <typename T> struct GradAcc {
    T u[3], A[3], M[9];
};

template <typename T>
__device__ __forceinline__ void kernel_KF(T r2, T sigma, T &K, T &F);

template <> __device__ __forceinline__ void kernel_KF<double>(double r2, double sigma, double &K, double &F)
{
    const double c = 0.79788456080286535588;
    double s2 = sigma * sigma, x = r2 / s2;
    if (x < 0.25) {
        double kk = 0.0, ff = 0.0, xp = 1.0, xm1 = 1.0, fact = 1.0;
        for (int q = 0; q < 16; ++q) {
            double den = fact * (2 * q + 3);
            kk += (q & 1) ? -xp / den : xp / den;
            if (q >= 1) ff += (q & 1) ? -2.0 * q * xm1 / den : 2.0 * q * xm1 / den;
            xm1 = xp;
            xp *= x;
            fact *= 2.0 * (q + 1);
        }
        K = c / (s2 * sigma) * kk;
        F = c / (s2 * s2 * sigma) * ff;
    } else {
        double r = sqrt(r2), rho = r / sigma, e = exp(-0.5 * x);
        double q = erf(rho * 0.70710678118654752440) - c * rho * e;
        K = q / (r2 * r);
        F = (c * e / (s2 * sigma) - 3.0 * K) / r2;
    }
}

template <> __device__ __forceinline__ void kernel_KF<float>(float r2, float sigma, float &K, float &F)
{
    const float c = 0.79788456080286535588f;
    float s2 = sigma * sigma, x = r2 / s2;
    if (x < 0.25f) {
        K = c / (s2 * sigma) * series_k<float>(x);
        F = c / (s2 * s2 * sigma) * series_f<float>(x);
    } else {
        float rinv = rsqrt_approx(r2), r = r2 * rinv;
        float e = ex2_approx(-0.72134752044448170368f * x);  // exp(-x/2) = 2^(-x log2(e)/2)
        float t = rcp_approx(fmaf(r, 0.3275911f * 0.70710678118654752440f / sigma, 1.0f));
        float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                              0.254829592f);
        float q = fmaf(-e, fmaf(c / sigma, r, poly), 1.0f);
        float rinv2 = rinv * rinv;
        K = q * rinv2 * rinv;
        F = rinv2 * (c * e / (s2 * sigma) - 3.0f * K);
    }
}

constexpr int PG_BS = 64;

template <typename T>
__global__ void __launch_bounds__(PG_BS) k_p2p_grad(const typename V4<T>::type *__restrict__ xs,
                                                    const typename V4<T>::type *__restrict__ gs,
                                                    const int *__restrict__ ls, int nside, int log2n, int R, int direct_K,
                                                    T leaf_w, T sigma, T L, const T *__restrict__ ufar,
                                                    const T *__restrict__ gfar, const int *__restrict__ perm,
                                                    T *__restrict__ u_out, T *__restrict__ g_out)
{
    typedef typename V4<T>::type T4;
    __shared__ T4 sx[PG_BS];
    __shared__ T4 sg[PG_BS];
    const int leaf = blockIdx.x;
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const int tb = ls[leaf], te = ls[leaf + 1];
    const T zx = (cx + T(0.5)) * leaf_w, zy = (cy + T(0.5)) * leaf_w, zz = (cz + T(0.5)) * leaf_w;
    for (int t0 = tb + blockIdx.y * PG_BS; t0 < te; t0 += gridDim.y * PG_BS) {
        const int ti = t0 + threadIdx.x;
        const bool active = ti < te;
        T4 xi = active ? xs[ti] : make_v4<T>(zx, zy, zz, T(0));
        T xi0 = xi.x - zx, xi1 = xi.y - zy, xi2 = xi.z - zz;  // leaf-relative
        GradAcc<T> a;
        for (int q = 0; q < 3; ++q) a.u[q] = a.A[q] = 0;
        for (int q = 0; q < 9; ++q) a.M[q] = 0;
        int lo[3], hi[3];
        const int cc[3] = {cx, cy, cz};
        for (int d = 0; d < 3; ++d) {
            lo[d] = direct_K >= 0 ? -cc[d] - direct_K * nside : -R;
            hi[d] = direct_K >= 0 ? nside - 1 - cc[d] + direct_K * nside : R;
        }
        for (int ox = lo[0]; ox <= hi[0]; ++ox)
            for (int oy = lo[1]; oy <= hi[1]; ++oy)
                for (int oz = lo[2]; oz <= hi[2]; ++oz) {
                    int nx = cx + ox, ny = cy + oy, nz = cz + oz;
                    int sl = ((nx & (nside - 1)) * nside + (ny & (nside - 1))) * nside + (nz & (nside - 1));
                    T o0 = L * (T)(nx >> log2n) - zx, o1 = L * (T)(ny >> log2n) - zy, o2 = L * (T)(nz >> log2n) - zz;
                    const bool own = ox == 0 && oy == 0 && oz == 0;  // own leaf, primary image: skip j = i
                    int sb = ls[sl], se = ls[sl + 1];
                    for (int s0 = sb; s0 < se; s0 += PG_BS) {
                        int cnt = min(PG_BS, se - s0);
                        __syncthreads();
                        if (threadIdx.x < cnt) {
                            T4 x = xs[s0 + threadIdx.x];
                            sx[threadIdx.x] = make_v4<T>(x.x + o0, x.y + o1, x.z + o2, T(0));
                            sg[threadIdx.x] = gs[s0 + threadIdx.x];
                        }
                        __syncthreads();
                        for (int j = 0; j < cnt; ++j) {
                            if (own && s0 + j == ti) continue;
                            T4 xj = sx[j], gj = sg[j];
                            T r0 = xi0 - xj.x, r1 = xi1 - xj.y, r2c = xi2 - xj.z;
                            T r2 = r0 * r0 + r1 * r1 + r2c * r2c;
                            T K, F;
                            kernel_KF<T>(r2, sigma, K, F);
                            T W0 = gj.y * r2c - gj.z * r1, W1 = gj.z * r0 - gj.x * r2c, W2 = gj.x * r1 - gj.y * r0;
                            a.u[0] += K * W0;
                            a.u[1] += K * W1;
                            a.u[2] += K * W2;
                            a.A[0] += K * gj.x;
                            a.A[1] += K * gj.y;
                            a.A[2] += K * gj.z;
                            T FW0 = F * W0, FW1 = F * W1, FW2 = F * W2;
                            a.M[0] += FW0 * r0; a.M[1] += FW0 * r1; a.M[2] += FW0 * r2c;
                            a.M[3] += FW1 * r0; a.M[4] += FW1 * r1; a.M[5] += FW1 * r2c;
                            a.M[6] += FW2 * r0; a.M[7] += FW2 * r1; a.M[8] += FW2 * r2c;
                        }
                    }
                }
        if (!active) continue;
        const T f = T(0.0795774715459476679);
        // G_ak = eps_abk A_b + M_ak
        T G[9];
        G[0] = a.M[0];
        G[1] = a.M[1] - a.A[2];
        G[2] = a.M[2] + a.A[1];
        G[3] = a.M[3] + a.A[2];
        G[4] = a.M[4];
        G[5] = a.M[5] - a.A[0];
        G[6] = a.M[6] - a.A[1];
        G[7] = a.M[7] + a.A[0];
        G[8] = a.M[8];
        int64_t o = perm[ti];
        for (int q = 0; q < 3; ++q) u_out[3 * o + q] = f * a.u[q] + (ufar ? ufar[3 * (int64_t)ti + q] : T(0));
        for (int q = 0; q < 9; ++q) g_out[9 * o + q] = f * G[q] + (gfar ? gfar[9 * (int64_t)ti + q] : T(0));
    }
}

int launch_p2p_grad(Ctx *c, int R, double sigma, const void *ufar, const void *gfar, void *u_out, void *g_out,
                    int direct_K)
{
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    int chunks = (c->max_leaf + PG_BS - 1) / PG_BS;
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    dim3 grid((unsigned)c->nleaf, (unsigned)chunks);
    if (c->f64)
        k_p2p_grad<double><<<grid, PG_BS, 0, c->stream>>>((const dvec4 *)c->xs.p, (const dvec4 *)c->gs.p,
                                                         (const int *)c->leaf_start.p, c->nside, log2n, R, direct_K,
                                                         c->leaf_w, sigma, c->cfg.box, (const double *)ufar,
                                                         (const double *)gfar, (const int *)c->perm.p,
                                                         (double *)u_out, (double *)g_out);
    else
        k_p2p_grad<float><<<grid, PG_BS, 0, c->stream>>>((const float4 *)c->xs.p, (const float4 *)c->gs.p,
                                                        (const int *)c->leaf_start.p, c->nside, log2n, R, direct_K,
                                                        (float)c->leaf_w, (float)sigma, (float)c->cfg.box,
                                                        (const float *)ufar, (const float *)gfar,
                                                        (const int *)c->perm.p, (float *)u_out, (float *)g_out);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

// dx_m = G1_m^T w_m + G2_m^T gamma_m (all arrays in caller order)
template <typename T>
__global__ void k_adjoint_combine(int64_t n, const T *__restrict__ G1, const T *__restrict__ w,
                                  const T *__restrict__ G2, const T *__restrict__ g, const T *__restrict__ extra,
                                  T *__restrict__ dx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 3; ++k) {
        T s = extra ? extra[3 * i + k] : T(0);
        for (int a = 0; a < 3; ++a) s += G1[9 * i + 3 * a + k] * w[3 * i + a] + G2[9 * i + 3 * a + k] * g[3 * i + a];
        dx[3 * i + k] = s;
    }
}

int launch_adjoint_combine(Ctx *c, const void *G1, const void *w, const void *G2, const void *gamma, const void *extra,
                           void *dx)
{
    int nb = (int)((c->n + 255) / 256);
    if (c->f64)
        k_adjoint_combine<double><<<nb, 256, 0, c->stream>>>(c->n, (const double *)G1, (const double *)w,
                                                            (const double *)G2, (const double *)gamma,
                                                            (const double *)extra, (double *)dx);
    else
        k_adjoint_combine<float><<<nb, 256, 0, c->stream>>>(c->n, (const float *)G1, (const float *)w,
                                                           (const float *)G2, (const float *)gamma,
                                                           (const float *)extra, (float *)dx);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

}  // namespace vfmm

// Near-field P2P of the Gaussian-regularised Biot-Savart kernel and its stretching term.
//
// For every target i and every source j in the (2R+1)^3 neighbour leaves of i's leaf
// (periodically wrapped, each with its image shift), excluding j = i:
//   u_i += K(r) gamma_j x r,                         Eq. (biotsavart)
//   S_i += K(r) gamma_j x gamma_i + F(r)(gamma_i.r)(gamma_j x r)      Eq. (stretching)
//   K = q(rho)/(4 pi r^3),  F = K'(r)/r,  q from Eq. (cutoff).
// The near field is "solved exactly" (Section 3.1): the full smoothed kernel, no expansion.
//
// Design: one block per target leaf (and target chunk); each thread owns one target and
// keeps nine FP32 accumulators (u, A = sum K gamma_j, B = sum F (gamma_i.r) gamma_j x r,
// S = A x gamma_i + B); sources of one neighbour leaf are staged in shared memory and read
// as warp-wide broadcasts.  The image shift is applied once per neighbour leaf to the
// target position.  FP32 math:
//   * 1/r from rsqrt, exp(-rho^2/2) from ex2, both single MUFU instructions;
//   * erf(rho/sqrt2) by Abramowitz & Stegun 7.1.26 (Hastings' rational approximation,
//     |error| <= 1.5e-7), which needs exactly the exp(-rho^2/2) already computed;
//   * for rho < 0.5 the Taylor series of q/rho^3 and of K'/r in rho^2, which avoids the
//     cancellation of q ~ rho^3 and the 1/r^5 of F, and gives the exact self-pair limit
//     (K finite, r = 0 so every self term vanishes).
// The epilogue adds the far field computed by L2P and scatters u, S to caller order.
#include "common.cuh"
#include "vfmm_internal.h"

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

// The same interaction without the small-rho series (valid when every pair of the two leaves
// has rho >= 0.5, so r > 0 and the closed form has no cancellation trouble).
__device__ __forceinline__ void pair_f32_smooth(const P2PConst &k, float xi0, float xi1, float xi2, float gi0,
                                                float gi1, float gi2, float4 xj, float4 gj, Acc &acc)
{
    float dx = xi0 - xj.x, dy = xi1 - xj.y, dz = xi2 - xj.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float e = ex2_approx(r2 * k.ce);
    float rinv = rsqrt_approx(r2);
    float r = r2 * rinv;
    float t = rcp_approx(fmaf(r, k.ct, 1.0f));
    float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                          0.254829592f);
    float q = fmaf(-e, fmaf(k.cq, r, poly), 1.0f);
    float rinv2 = rinv * rinv;
    float K = q * (rinv2 * rinv);
    float F = rinv2 * fmaf(-3.0f, K, k.cf * e);
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

// Leaves whose closest pair has rho >= 6.5: q = 1 - O(1e-9) and the Gaussian term of F is
// O(1e-7) relative, so the kernel is the singular Biot-Savart kernel to FP32 rounding
// (K = 1/r^3, F = -3/r^5, before the common 1/(4 pi)).
__device__ __forceinline__ void pair_f32_singular(float xi0, float xi1, float xi2, float gi0, float gi1, float gi2,
                                                  float4 xj, float4 gj, Acc &acc)
{
    float dx = xi0 - xj.x, dy = xi1 - xj.y, dz = xi2 - xj.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float rinv = rsqrt_approx(r2);
    float rinv2 = rinv * rinv;
    float K = rinv2 * rinv;
    float F = -3.0f * K * rinv2;
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

template <int MODE>
__device__ __forceinline__ void source_tile(const P2PConst &kc, float xi0, float xi1, float xi2, float4 gi,
                                            const float4 *sx, const float4 *sg, int cnt, Acc &acc)
{
    int j = 0;
    for (; j + 4 <= cnt; j += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (MODE == 0) pair_f32(kc, xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j + u], sg[j + u], acc);
            else if (MODE == 1) pair_f32_smooth(kc, xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j + u], sg[j + u], acc);
            else pair_f32_singular(xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j + u], sg[j + u], acc);
        }
    }
    for (; j < cnt; ++j) {
        if (MODE == 0) pair_f32(kc, xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j], sg[j], acc);
        else if (MODE == 1) pair_f32_smooth(kc, xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j], sg[j], acc);
        else pair_f32_singular(xi0, xi1, xi2, gi.x, gi.y, gi.z, sx[j], sg[j], acc);
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

__global__ void __launch_bounds__(P2P_BS) k_p2p_f32(const float4 *__restrict__ xs, const float4 *__restrict__ gs,
                                                    const int *__restrict__ ls, const float4 *__restrict__ bbox,
                                                    int nside, int log2n, int R, P2PConst kc,
                                                    const float *__restrict__ ufar, const float *__restrict__ sfar,
                                                    const int *__restrict__ perm, float *__restrict__ u_out,
                                                    float *__restrict__ s_out)
{
    __shared__ float4 sx[P2P_BS];
    __shared__ float4 sg[P2P_BS];
    const int leaf = blockIdx.x;
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const int tb = ls[leaf], te = ls[leaf + 1];
    const float Lf = (float)kc.L;
    const float4 tlo = bbox[2 * leaf], thi = bbox[2 * leaf + 1];
    for (int t0 = tb + blockIdx.y * P2P_BS; t0 < te; t0 += gridDim.y * P2P_BS) {
        const int ti = t0 + threadIdx.x;
        const bool active = ti < te;
        float4 xi = active ? xs[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 gi = active ? gs[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
        Acc acc = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int ox = -R; ox <= R; ++ox)
            for (int oy = -R; oy <= R; ++oy)
                for (int oz = -R; oz <= R; ++oz) {
                    int nx = cx + ox, ny = cy + oy, nz = cz + oz;
                    int sl = ((nx & (nside - 1)) * nside + (ny & (nside - 1))) * nside + (nz & (nside - 1));
                    // image shift of this neighbour; the target is moved by minus the shift
                    float shx = Lf * (float)(nx >> log2n), shy = Lf * (float)(ny >> log2n), shz = Lf * (float)(nz >> log2n);
                    float xi0 = xi.x - shx, xi1 = xi.y - shy, xi2 = xi.z - shz;
                    // closest approach of the two leaf boxes selects the inner loop (block-uniform)
                    float4 slo = bbox[2 * sl], shi = bbox[2 * sl + 1];
                    float gx = fmaxf(0.f, fmaxf(slo.x + shx - thi.x, tlo.x - shi.x - shx));
                    float gy = fmaxf(0.f, fmaxf(slo.y + shy - thi.y, tlo.y - shi.y - shy));
                    float gz = fmaxf(0.f, fmaxf(slo.z + shz - thi.z, tlo.z - shi.z - shz));
                    float d2 = gx * gx + gy * gy + gz * gz;
                    const int mode = d2 >= kc.d2_singular ? 2 : (d2 >= kc.d2_series ? 1 : 0);
                    int sb = ls[sl], se = ls[sl + 1];
                    for (int s0 = sb; s0 < se; s0 += P2P_BS) {
                        int cnt = min(P2P_BS, se - s0);
                        __syncthreads();
                        if (threadIdx.x < cnt) {
                            sx[threadIdx.x] = xs[s0 + threadIdx.x];
                            sg[threadIdx.x] = gs[s0 + threadIdx.x];
                        }
                        __syncthreads();
                        if (mode == 2) source_tile<2>(kc, xi0, xi1, xi2, gi, sx, sg, cnt, acc);
                        else if (mode == 1) source_tile<1>(kc, xi0, xi1, xi2, gi, sx, sg, cnt, acc);
                        else source_tile<0>(kc, xi0, xi1, xi2, gi, sx, sg, cnt, acc);
                    }
                }
        if (active) {
            float s0 = fmaf(acc.a1, gi.z, fmaf(-acc.a2, gi.y, acc.b0));
            float s1 = fmaf(acc.a2, gi.x, fmaf(-acc.a0, gi.z, acc.b1));
            float s2 = fmaf(acc.a0, gi.y, fmaf(-acc.a1, gi.x, acc.b2));
            float u0 = acc.u0 * INV_4PI_F, u1 = acc.u1 * INV_4PI_F, u2 = acc.u2 * INV_4PI_F;
            s0 *= INV_4PI_F;
            s1 *= INV_4PI_F;
            s2 *= INV_4PI_F;
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
}

__global__ void __launch_bounds__(P2P_BS) k_p2p_f64(const dvec4 *__restrict__ xs, const dvec4 *__restrict__ gs,
                                                    const int *__restrict__ ls, int nside, int log2n, int R,
                                                    double sigma, double L, const double *__restrict__ ufar,
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
        for (int ox = -R; ox <= R; ++ox)
            for (int oy = -R; oy <= R; ++oy)
                for (int oz = -R; oz <= R; ++oz) {
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

int launch_p2p(Ctx *c, int R, double sigma, const void *ufar, const void *sfar, void *u_out, void *s_out, int)
{
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    int chunks = (c->max_leaf + P2P_BS - 1) / P2P_BS;
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    dim3 grid((unsigned)c->nleaf, (unsigned)chunks);
    if (c->f64) {
        k_p2p_f64<<<grid, P2P_BS, 0, c->stream>>>((const dvec4 *)c->xs.p, (const dvec4 *)c->gs.p,
                                                  (const int *)c->leaf_start.p, c->nside, log2n, R, sigma,
                                                  c->cfg.box, (const double *)ufar, (const double *)sfar,
                                                  (const int *)c->perm.p, (double *)u_out, (double *)s_out);
    } else {
        P2PConst kc;
        kc.sigma = sigma;
        kc.L = c->cfg.box;
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
        kc.d2_series = (float)(0.36 * sigma * sigma);      // (0.6 sigma)^2: margin over rho = 0.5
        kc.d2_singular = (float)(42.25 * sigma * sigma);   // (6.5 sigma)^2
        k_p2p_f32<<<grid, P2P_BS, 0, c->stream>>>((const float4 *)c->xs.p, (const float4 *)c->gs.p,
                                                  (const int *)c->leaf_start.p, (const float4 *)c->bbox.p,
                                                  c->nside, log2n, R, kc,
                                                  (const float *)ufar, (const float *)sfar, (const int *)c->perm.p,
                                                  (float *)u_out, (float *)s_out);
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
    float4 *scratch;
    {
        // one-time set-up per device: the host-side symbol is only a stand-in, so look up the
        // array's device address with that device current
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
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

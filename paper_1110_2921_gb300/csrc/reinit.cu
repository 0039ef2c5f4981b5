// Reinitialisation of the particle set onto a lattice (Section 2.2, RBF interpolation;
// Section 5.3 for the initial guess gamma = omega dx^3).
//
// 1. omega(x_g) = sum_j gamma_j zeta_sigma(x_g - x_j) at the lattice points, zeta the Gaussian
//    basis of Eq. (gaussian), from the octree of the old particles (leaf pairs farther than
//    6 sigma apart are skipped: zeta(6 sigma)/zeta(0) = 1.5e-8).
// 2. gamma' minimises 0.5 |Z gamma' - omega|^2 by steepest descent with exact line search,
//    Z_gk = zeta_sigma0(x_g - x_k) between lattice points.  On the lattice Z is a product of
//    three periodic 1-D Gaussian convolutions (zeta factorises per axis), so Z v is three
//    (2 R_t + 1)-tap stencil passes, R_t = ceil(6 sigma0 / h), instead of a 3-D pair sum.
//    Step sizes are formed on the device; no host round trip per iteration.
#include "common.cuh"
#include "vfmm_internal.h"

#include <cmath>

namespace vfmm {

constexpr int RG_MAXTAPS = 65;
struct ConvW {
    double w[RG_MAXTAPS];
    int R;
};

template <typename T>
__global__ void __launch_bounds__(256) k_gauss_to_lattice(const typename V4<T>::type *__restrict__ xs,
                                                          const typename V4<T>::type *__restrict__ gs,
                                                          const int *__restrict__ ls, const float4 *__restrict__ bbox,
                                                          int nside, int log2n, int R, int npl1, int m, T h, T L,
                                                          T sigma, T *__restrict__ omega)
{
    typedef typename V4<T>::type T4;
    __shared__ T4 sx[128];
    __shared__ T4 sg[128];
    const int leaf = blockIdx.x;
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const T w = L / (T)nside;
    const T inv2s2 = T(0.5) / (sigma * sigma);
    const T norm = pow(T(2) * T(3.14159265358979323846) * sigma * sigma, T(-1.5));
    const T cut2 = T(36) * sigma * sigma;
    // box of this leaf's lattice points
    const T tlo[3] = {cx * w + T(0.5) * h, cy * w + T(0.5) * h, cz * w + T(0.5) * h};
    const T thi[3] = {(cx + 1) * w - T(0.5) * h, (cy + 1) * w - T(0.5) * h, (cz + 1) * w - T(0.5) * h};
    const int ntl = npl1 * npl1 * npl1;
    for (int t0 = 0; t0 < ntl; t0 += blockDim.x) {
        const int tl = t0 + threadIdx.x;
        const bool active = tl < ntl;
        int lx = tl / (npl1 * npl1), ly = (tl / npl1) % npl1, lz = tl % npl1;
        int gx = cx * npl1 + lx, gy = cy * npl1 + ly, gz = cz * npl1 + lz;
        T px = (gx + T(0.5)) * h, py = (gy + T(0.5)) * h, pz = (gz + T(0.5)) * h;
        T a0 = 0, a1 = 0, a2 = 0;
        for (int ox = -R; ox <= R; ++ox)
            for (int oy = -R; oy <= R; ++oy)
                for (int oz = -R; oz <= R; ++oz) {
                    int nx = cx + ox, ny = cy + oy, nz = cz + oz;
                    int sl = ((nx & (nside - 1)) * nside + (ny & (nside - 1))) * nside + (nz & (nside - 1));
                    T sh[3] = {L * (T)(nx >> log2n), L * (T)(ny >> log2n), L * (T)(nz >> log2n)};
                    float4 blo = bbox[2 * sl], bhi = bbox[2 * sl + 1];
                    T slo[3] = {(T)blo.x, (T)blo.y, (T)blo.z}, shi[3] = {(T)bhi.x, (T)bhi.y, (T)bhi.z};
                    T d2 = 0;
                    for (int d = 0; d < 3; ++d) {
                        T gap = slo[d] + sh[d] - thi[d];
                        T gap2 = tlo[d] - shi[d] - sh[d];
                        gap = gap > gap2 ? gap : gap2;
                        if (gap > 0) d2 += gap * gap;
                    }
                    if (d2 > cut2) continue;  // block-uniform
                    int sb = ls[sl], se = ls[sl + 1];
                    for (int s0 = sb; s0 < se; s0 += 128) {
                        int cnt = min(128, se - s0);
                        __syncthreads();
                        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
                            T4 x = xs[s0 + j];
                            sx[j] = make_v4<T>(x.x + sh[0], x.y + sh[1], x.z + sh[2], T(0));
                            sg[j] = gs[s0 + j];
                        }
                        __syncthreads();
                        for (int j = 0; j < cnt; ++j) {
                            T4 xj = sx[j], gj = sg[j];
                            T dx = px - xj.x, dy = py - xj.y, dz = pz - xj.z;
                            T e = exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
                            a0 += e * gj.x;
                            a1 += e * gj.y;
                            a2 += e * gj.z;
                        }
                    }
                }
        if (active) {
            int64_t g = ((int64_t)gx * m + gy) * m + gz;
            omega[3 * g + 0] = norm * a0;
            omega[3 * g + 1] = norm * a1;
            omega[3 * g + 2] = norm * a2;
        }
    }
}

// one axis of the separable lattice Gaussian: out(i) = sum_d w_d in(i + d e_axis), periodic
template <typename T>
__global__ void k_gauss_conv_axis(int m, int axis, ConvW cw, const T *__restrict__ in, T *__restrict__ out)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)m * m * m;
    if (idx >= total) return;
    int i = (int)(idx / ((int64_t)m * m)), j = (int)((idx / m) % m), k = (int)(idx % m);
    T a0 = 0, a1 = 0, a2 = 0;
    for (int d = -cw.R; d <= cw.R; ++d) {
        int ii = i, jj = j, kk = k;
        if (axis == 0) ii = ((i + d) % m + m) % m;
        else if (axis == 1) jj = ((j + d) % m + m) % m;
        else kk = ((k + d) % m + m) % m;
        int64_t s = ((int64_t)ii * m + jj) * m + kk;
        T wd = (T)cw.w[d + cw.R];
        a0 += wd * in[3 * s + 0];
        a1 += wd * in[3 * s + 1];
        a2 += wd * in[3 * s + 2];
    }
    out[3 * idx + 0] = a0;
    out[3 * idx + 1] = a1;
    out[3 * idx + 2] = a2;
}

template <typename T>
__global__ void k_scale(int64_t n3, T c, const T *__restrict__ in, T *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) out[i] = c * in[i];
}

// out[0] += a.b, out[1] += b.b  (FP64)
template <typename T>
__global__ void k_dot2(int64_t n3, const T *__restrict__ a, const T *__restrict__ b, double *__restrict__ out)
{
    double ab = 0, bb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        double av = a[i], bv = b[i];
        ab += av * bv;
        bb += bv * bv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ab += __shfl_xor_sync(0xffffffffu, ab, o);
        bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], ab);
        atomicAdd(&out[1], bb);
    }
}

// alpha = (r.q)/(q.q); g += alpha d; r -= alpha q
template <typename T>
__global__ void k_sd_update(int64_t n3, const double *__restrict__ dots, T *__restrict__ g, T *__restrict__ r,
                            const T *__restrict__ d, const T *__restrict__ q)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    double qq = dots[1];
    T alpha = qq > 0.0 ? (T)(dots[0] / qq) : T(0);
    g[i] += alpha * d[i];
    r[i] -= alpha * q[i];
}

template <typename T>
__global__ void k_lattice_positions(int m, T h, T *__restrict__ x)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)m * m * m;
    if (idx >= total) return;
    int i = (int)(idx / ((int64_t)m * m)), j = (int)((idx / m) % m), k = (int)(idx % m);
    x[3 * idx + 0] = (i + T(0.5)) * h;
    x[3 * idx + 1] = (j + T(0.5)) * h;
    x[3 * idx + 2] = (k + T(0.5)) * h;
}

template <typename T> static int reinit_impl(Ctx *c, int m, double sigma, double sigma0, int iters, int R,
                                              void *x_new, void *g_new, double *residual)
{
    cudaStream_t st = c->stream;
    const double L = c->cfg.box, h = L / m;
    const int64_t np = (int64_t)m * m * m, n3 = 3 * np;
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    const int npl1 = m >> log2n;
    T *om = (T *)c->rg_om.p, *r = (T *)c->rg_r.p, *d = (T *)c->rg_d.p, *q = (T *)c->rg_q.p;
    T *t1 = (T *)c->rg_t1.p, *t2 = (T *)c->rg_t2.p, *g = (T *)g_new;
    double *dots = (double *)c->rg_dots.p;
    int tpb = npl1 * npl1 * npl1;
    tpb = tpb > 256 ? 256 : (tpb < 32 ? 32 : ((tpb + 31) / 32) * 32);
    k_gauss_to_lattice<T><<<(unsigned)c->nleaf, tpb, 0, st>>>(
        (const typename V4<T>::type *)c->xs.p, (const typename V4<T>::type *)c->gs.p, (const int *)c->leaf_start.p,
        (const float4 *)c->bbox.p, c->nside, log2n, R, npl1, m, (T)h, (T)L, (T)sigma, om);
    VFMM_CUDA_CHECK_LAUNCH(c);
    ConvW cw;
    cw.R = (int)std::ceil(6.0 * sigma0 / h);
    if (cw.R < 1) cw.R = 1;
    if (2 * cw.R + 1 > RG_MAXTAPS) {
        c->last_error = "sigma_new / lattice spacing too large (more than 32 taps per side)";
        return VFMM_ERR_UNSUPPORTED;
    }
    const double w1 = 1.0 / std::sqrt(2.0 * M_PI * sigma0 * sigma0);
    for (int k = -cw.R; k <= cw.R; ++k) cw.w[k + cw.R] = w1 * std::exp(-0.5 * (k * h) * (k * h) / (sigma0 * sigma0));
    const int nb = (int)((np + 255) / 256), nb3 = (int)((n3 + 255) / 256);
    auto applyZ = [&](const T *in, T *out) {
        k_gauss_conv_axis<T><<<nb, 256, 0, st>>>(m, 2, cw, in, t1);
        k_gauss_conv_axis<T><<<nb, 256, 0, st>>>(m, 1, cw, t1, t2);
        k_gauss_conv_axis<T><<<nb, 256, 0, st>>>(m, 0, cw, t2, out);
        c->launches += 3;
    };
    k_scale<T><<<nb3, 256, 0, st>>>(n3, (T)(h * h * h), om, g);
    applyZ(g, d);
    k_scale<T><<<nb3, 256, 0, st>>>(n3, T(-1), d, r);
    int rc = launch_axpy3(c, np, om, r, nullptr, 1.0, 0.0, r);  // r = omega - Z g
    if (rc) return rc;
    const int nbd = 4 * 152;
    for (int it = 0; it < iters; ++it) {
        applyZ(r, d);
        applyZ(d, q);
        cudaMemsetAsync(dots, 0, 2 * sizeof(double), st);
        k_dot2<T><<<nbd, 256, 0, st>>>(n3, r, q, dots);
        k_sd_update<T><<<nb3, 256, 0, st>>>(n3, dots, g, r, d, q);
        c->launches += 2;
    }
    cudaMemsetAsync(dots, 0, 4 * sizeof(double), st);
    k_dot2<T><<<nbd, 256, 0, st>>>(n3, om, r, dots);       // dots[1] = r.r
    k_dot2<T><<<nbd, 256, 0, st>>>(n3, r, om, dots + 2);   // dots[3] = om.om
    k_lattice_positions<T><<<nb, 256, 0, st>>>(m, (T)h, (T *)x_new);
    c->launches += 5;
    VFMM_CUDA_CHECK_LAUNCH(c);
    double hd[4];
    cudaError_t e = cudaMemcpyAsync(hd, dots, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        c->last_error = std::string("reinit: ") + cudaGetErrorString(e);
        return VFMM_ERR_CUDA;
    }
    if (residual) *residual = hd[3] > 0 ? std::sqrt(hd[1] / hd[3]) : 0.0;
    return VFMM_OK;
}

int launch_reinit(Ctx *c, int m, double sigma, double sigma0, int iters, int R, void *x_new, void *g_new,
                  double *residual)
{
    if (c->f64) return reinit_impl<double>(c, m, sigma, sigma0, iters, R, x_new, g_new, residual);
    return reinit_impl<float>(c, m, sigma, sigma0, iters, R, x_new, g_new, residual);
}

}  // namespace vfmm

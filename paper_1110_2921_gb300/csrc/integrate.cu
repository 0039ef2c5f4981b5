// Time integration of the vortex method and FP64 diagnostics.
//
// Section 2.2: positions move with the velocity (Eq. convection), strengths change by the
// stretching term (Eq. stretching) and the core variance grows as d sigma^2/dt = 2 nu
// (Eq. csm), all simultaneously.  vfmm_rk_step takes one explicit trapezoid (Heun) step with
// two FMM evaluations; the paper's own integrator is forward Euler (Section 4.1).
#include "common.cuh"
#include "vfmm_internal.h"

namespace vfmm {

// out = a + c (b + d) (d may be NULL); wrap_L > 0 wraps the result into [0, L)
template <typename T>
__global__ void k_axpy3(int64_t n3, const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ d, T c,
                        T wrap_L, T *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    T v = b[i] + (d ? d[i] : T(0));
    T r = a[i] + c * v;
    if (wrap_L > T(0)) r = wrap_coord<T>(r, wrap_L, T(1) / wrap_L);
    out[i] = r;
}

int launch_axpy3(Ctx *c, int64_t n, const void *a, const void *b, const void *d, double coef, double wrap_L, void *out)
{
    int64_t n3 = 3 * n;
    int nb = (int)((n3 + 255) / 256);
    if (c->f64)
        k_axpy3<double><<<nb, 256, 0, c->stream>>>(n3, (const double *)a, (const double *)b, (const double *)d, coef,
                                                   wrap_L, (double *)out);
    else
        k_axpy3<float><<<nb, 256, 0, c->stream>>>(n3, (const float *)a, (const float *)b, (const float *)d,
                                                  (float)coef, (float)wrap_L, (float *)out);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

// FP64 sums: gamma (3), x cross gamma (3), |u|^2, |gamma|^2
template <typename T>
__global__ void k_diag(int64_t n, const T *__restrict__ x, const T *__restrict__ g, const T *__restrict__ u,
                       double *__restrict__ out)
{
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        double g0 = g[3 * i], g1 = g[3 * i + 1], g2 = g[3 * i + 2];
        v[0] += g0;
        v[1] += g1;
        v[2] += g2;
        v[3] += x1 * g2 - x2 * g1;
        v[4] += x2 * g0 - x0 * g2;
        v[5] += x0 * g1 - x1 * g0;
        if (u) {
            double u0 = u[3 * i], u1 = u[3 * i + 1], u2 = u[3 * i + 2];
            v[6] += u0 * u0 + u1 * u1 + u2 * u2;
        }
        v[7] += g0 * g0 + g1 * g1 + g2 * g2;
    }
    for (int k = 0; k < 8; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 8; ++k) atomicAdd(&out[k], v[k]);
}

int launch_diag(Ctx *c, int64_t n, const void *x, const void *g, const void *u, double *out_dev)
{
    int nb = (int)std::min<int64_t>((n + 255) / 256, 4 * 152);
    if (nb < 1) nb = 1;
    if (c->f64)
        k_diag<double><<<nb, 256, 0, c->stream>>>(n, (const double *)x, (const double *)g, (const double *)u, out_dev);
    else
        k_diag<float><<<nb, 256, 0, c->stream>>>(n, (const float *)x, (const float *)g, (const float *)u, out_dev);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

}  // namespace vfmm

// Turbulence diagnostics of Section 5.2: the energy spectrum of a velocity field sampled on
// the lattice (3-D FFT of the lattice velocity, shell sums of 0.5 |u_hat|^2) and the
// skewness / flatness F_n = mean(u_x^n) / mean(u_x^2)^(n/2) of the velocity derivatives.
// All in FP64.
//
// FFT: the three components are copied to FP64 complex arrays [c][ix][iy][iz]; each axis is
// transformed by one block per line, a radix-2 decimation-in-time transform of the whole
// line in shared memory (bit-reversed load, log2 n butterfly stages, twiddles from sincospi).
#include "common.cuh"
#include "vfmm_internal.h"

#include <algorithm>

namespace vfmm {

template <typename T>
__global__ void k_to_complex(int64_t m, const T *__restrict__ u, double2 *__restrict__ a)
{
    // u: (m, 3) lattice order -> a[c][m]
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) a[(int64_t)c * m + i] = make_double2((double)u[3 * i + c], 0.0);
}

__global__ void k_fft_axis(double2 *__restrict__ a, int n, int log2n, int axis)
{
    extern __shared__ double2 s[];
    const int64_t n2 = (int64_t)n * n, n3 = n2 * n;
    const int64_t line = blockIdx.x;  // 3 n^2 lines
    const int comp = (int)(line / n2);
    const int64_t r = line - comp * n2;
    const int i0 = (int)(r / n), i1 = (int)(r - (r / n) * n);
    int64_t base, stride;
    if (axis == 2) {  // z: (ix, iy) = (i0, i1)
        base = comp * n3 + ((int64_t)i0 * n + i1) * n;
        stride = 1;
    } else if (axis == 1) {  // y: (ix, iz) = (i0, i1)
        base = comp * n3 + (int64_t)i0 * n2 + i1;
        stride = n;
    } else {  // x: (iy, iz) = (i0, i1)
        base = comp * n3 + (int64_t)i0 * n + i1;
        stride = n2;
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) s[__brev((unsigned)t) >> (32 - log2n)] = a[base + t * stride];
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1;
        for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const int grp = b / half, pos = b - grp * half;
            const int i = grp * len + pos, j = i + half;
            double sn, cs;
            sincospi(-2.0 * pos / len, &sn, &cs);  // exp(-2 pi i pos / len)
            const double2 v = s[j], w0 = s[i];
            const double2 t = make_double2(cs * v.x - sn * v.y, cs * v.y + sn * v.x);
            s[i] = make_double2(w0.x + t.x, w0.y + t.y);
            s[j] = make_double2(w0.x - t.x, w0.y - t.y);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) a[base + t * stride] = s[t];
}

__global__ void k_shells(int n, const double2 *__restrict__ a, int kmax, double scale, double *__restrict__ E)
{
    // E[round |k|] += 0.5 scale sum_c |a_c(k)|^2 over the (signed) integer wave vectors
    extern __shared__ double bins[];
    for (int k = threadIdx.x; k <= kmax; k += blockDim.x) bins[k] = 0.0;
    __syncthreads();
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i / ((int64_t)n * n)), iy = (int)((i / n) % n), iz = (int)(i % n);
        const int kx = ix < n / 2 ? ix : ix - n, ky = iy < n / 2 ? iy : iy - n, kz = iz < n / 2 ? iz : iz - n;
        const int sh = (int)floor(sqrt((double)(kx * kx + ky * ky + kz * kz)) + 0.5);
        if (sh > kmax) continue;
        double e = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 v = a[(int64_t)c * n3 + i];
            e += v.x * v.x + v.y * v.y;
        }
        atomicAdd(&bins[sh], 0.5 * scale * e);
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= kmax; k += blockDim.x)
        if (bins[k] != 0.0) atomicAdd(&E[k], bins[k]);
}

int launch_spectrum(Ctx *c, int n, const void *u, int kmax, double2 *work, double *E_dev)
{
    int log2n = 0;
    while ((1 << log2n) < n) ++log2n;
    const int64_t m = (int64_t)n * n * n;
    const int nb = (int)((m + 255) / 256);
    if (c->f64)
        k_to_complex<double><<<nb, 256, 0, c->stream>>>(m, (const double *)u, work);
    else
        k_to_complex<float><<<nb, 256, 0, c->stream>>>(m, (const float *)u, work);
    VFMM_CUDA_CHECK_LAUNCH(c);
    const int bt = n / 2 < 256 ? (n / 2 > 32 ? n / 2 : 32) : 256;
    for (int axis = 0; axis < 3; ++axis) {
        k_fft_axis<<<(unsigned)(3 * (int64_t)n * n), bt, (size_t)n * sizeof(double2), c->stream>>>(work, n, log2n, axis);
        VFMM_CUDA_CHECK_LAUNCH(c);
    }
    cudaMemsetAsync(E_dev, 0, (size_t)(kmax + 1) * sizeof(double), c->stream);
    const double scale = 1.0 / ((double)m * (double)m);  // |u_hat|^2 with u_hat = n^-3 sum
    const int nbs = (int)std::min<int64_t>((m + 255) / 256, 4 * 152);
    k_shells<<<nbs, 256, (size_t)(kmax + 1) * sizeof(double), c->stream>>>(n, work, kmax, scale, E_dev);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

template <typename T>
__global__ void k_moments(int64_t n, const T *__restrict__ g, double *__restrict__ out)
{
    // sums of d^2, d^3, d^4 over the longitudinal derivatives du_a/dx_a (entries 0, 4, 8)
    double v2 = 0.0, v3 = 0.0, v4 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double d = (double)g[9 * i + 4 * a], d2 = d * d;
            v2 += d2;
            v3 += d2 * d;
            v4 += d2 * d2;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        v3 += __shfl_xor_sync(0xffffffffu, v3, o);
        v4 += __shfl_xor_sync(0xffffffffu, v4, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], v2);
        atomicAdd(&out[1], v3);
        atomicAdd(&out[2], v4);
    }
}

int launch_moments(Ctx *c, int64_t n, const void *g, double *out_dev)
{
    int nb = (int)std::min<int64_t>((n + 255) / 256, 4 * 152);
    if (nb < 1) nb = 1;
    if (c->f64)
        k_moments<double><<<nb, 256, 0, c->stream>>>(n, (const double *)g, out_dev);
    else
        k_moments<float><<<nb, 256, 0, c->stream>>>(n, (const float *)g, out_dev);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

}  // namespace vfmm

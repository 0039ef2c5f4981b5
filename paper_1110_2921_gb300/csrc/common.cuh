// Device-side helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vfmm {

struct __align__(32) dvec4 {
    double x, y, z, w;
};

template <typename T> struct V4;
template <> struct V4<float> { typedef float4 type; };
template <> struct V4<double> { typedef dvec4 type; };

template <typename T> __device__ __forceinline__ typename V4<T>::type make_v4(T x, T y, T z, T w)
{
    typename V4<T>::type v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = w;
    return v;
}

// Periodic wrap of one coordinate into [0, L): x - L floor(x / L), with L mapped to 0.
template <typename T> __device__ __forceinline__ T wrap_coord(T x, T L, T invL)
{
    T y = x - L * floor(x * invL);
    if (y >= L) y -= L;
    if (y < T(0)) y = T(0);
    return y;
}

__device__ __forceinline__ int imod_pow2(int v, int n) { return v & (n - 1); }

// An SM runs blocks of one shared-memory / L1 split at a time, so kernels that are meant to
// share SMs (the near-field P2P beside the far-field kernels) all ask for the largest shared
// carveout; otherwise an SM holding blocks of one split must drain before it takes the other.
template <typename K> inline void prefer_max_shared(K kernel)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    cudaGetLastError();
}
__device__ __forceinline__ int floordiv_pow2(int v, int log2n) { return v >> log2n; }

}  // namespace vfmm

#define VFMM_CUDA_CHECK_LAUNCH(ctx)                                                       \
    do {                                                                                  \
        (ctx)->launches++;                                                                \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            (ctx)->last_error = std::string("kernel launch: ") + cudaGetErrorString(e_);  \
            return VFMM_ERR_CUDA;                                                         \
        }                                                                                 \
    } while (0)

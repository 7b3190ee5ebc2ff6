// reduce_util.cuh -- warp and block reductions in a fixed order (bitwise
// reproducible for a given block size), shared by the membrane kernels.
#pragma once

namespace iblb {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o >= 1; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o >= 1; o >>= 1)
        v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o >= 1; o >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NV values per thread over a block of NT threads; kind[k]: 0 sum,
// 1 min, 2 max.  Result valid in thread 0.
template <int NV, int NT>
__device__ void block_reduce(double *v, const int *kind)
{
    __shared__ double sh[NV][NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < NV; ++k) {
        double x = kind[k] == 0 ? warp_sum(v[k]) : (kind[k] == 1 ? warp_min(v[k]) : warp_max(v[k]));
        if (lane == 0)
            sh[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) {
            double x = sh[k][0];
            for (int i = 1; i < NT / 32; ++i)
                x = kind[k] == 0 ? x + sh[k][i] : (kind[k] == 1 ? fmin(x, sh[k][i]) : fmax(x, sh[k][i]));
            v[k] = x;
        }
    __syncthreads();
}

}  // namespace iblb

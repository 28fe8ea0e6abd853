// Block-wide reductions shared by the one-block-per-walker complex128 kernels.
#pragma once

#include "complex_math.cuh"

namespace ftq {
namespace {

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ T block_sum(T v, T* sh) {
    // deterministic: fixed shuffle tree then fixed order over warps
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_down(v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        T acc = sh[0];
        for (int i = 1; i < (int)((blockDim.x + 31) >> 5); ++i) acc = acc + sh[i];
        sh[0] = acc;
    }
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

// argmax of val over the block; ties go to the lowest index.
__device__ int block_argmax(double val, int idx, double* shv, int* shi) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, val, o);
        int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { shv[wid] = val; shi[wid] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = shv[0];
        int bi = shi[0];
        for (int i = 1; i < (int)((blockDim.x + 31) >> 5); ++i)
            if (shv[i] > bv || (shv[i] == bv && shi[i] < bi)) { bv = shv[i]; bi = shi[i]; }
        shi[0] = bi;
    }
    __syncthreads();
    int r = shi[0];
    __syncthreads();
    return r;
}

}  // namespace
}  // namespace ftq

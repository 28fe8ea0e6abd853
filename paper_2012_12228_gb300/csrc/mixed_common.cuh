// Shared pieces of the mixed-precision chain: tf32 hi/lo splitting and the
// K-major plane layout of the chain matrix.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ftq {

__device__ __forceinline__ float tf32_rna(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// v ~= hi + lo with hi, lo both tf32 values (|v - hi - lo| <= 2^-22 |v|)
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
    hi = tf32_rna(v);
    lo = tf32_rna(v - hi);
}

// x * s for a scale s held in double: s is split into a float pair
// (hi + lo) so that the product carries no systematic rounding of s.  The
// kinetic factors multiply the chain on every slice; a float-rounded factor
// would bias ln D by n times its rounding error over a path of n slices.
struct ScaleF {
    float hi, lo;
    __device__ __forceinline__ explicit ScaleF(double s) {
        hi = (float)s;
        lo = (float)(s - (double)hi);
    }
    __device__ __forceinline__ explicit ScaleF(float2 p) : hi(p.x), lo(p.y) {}
    __device__ __forceinline__ float operator()(float x) const { return fmaf(lo, x, hi * x); }
};

// Chain layout (mixed): per walker two parts (tf32 hi, tf32 lo), each LDc
// rows of 2 Kp floats; row c holds column c of Y as [Re Y[0..Kp) | Im Y[0..Kp)].
// A row is one K-major operand row of the real-embedded product, so the
// tensor-core kernel reads it with TMA directly.
struct Planes {
    int Kp;
    size_t part;     // LDc * 2 Kp
    __device__ __forceinline__ float2 load(const float* w, int i, int c) const {
        size_t o = (size_t)c * (2 * Kp) + i;
        return make_float2(w[o] + w[part + o], w[o + Kp] + w[part + o + Kp]);
    }
    __device__ __forceinline__ void store(float* w, int i, int c, float2 v) const {
        size_t o = (size_t)c * (2 * Kp) + i;
        float h, l;
        split_tf32(v.x, h, l);
        w[o] = h;
        w[part + o] = l;
        split_tf32(v.y, h, l);
        w[o + Kp] = h;
        w[part + o + Kp] = l;
    }
};

}  // namespace ftq

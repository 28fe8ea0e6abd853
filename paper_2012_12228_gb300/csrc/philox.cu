// On-device auxiliary-field generator: Philox4x32-10 (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from
// its published definition, followed by the Box-Muller transform in FP64.
//
// One counter per pair of fields: (j, k, w, s) = (pair index alpha / 2,
// absolute slice index k (0-based), walker, system id); key = (low, high)
// 32-bit halves of the seed.  The four output words give two 53-bit uniforms
// u = ((hi << 32 | lo) >> 11 + 1/2) 2^-53 in (0, 1), and
// x_{2j} = r cos t, x_{2j+1} = r sin t with r = sqrt(-2 ln u1), t = 2 pi u2.
#include <cstdint>

#include "ftq_internal.h"

namespace ftq {
namespace {

constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;   // round multipliers
constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u; // key schedule increments
constexpr double kTwoPi = 6.283185307179586;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kMul0, c.x), lo0 = kMul0 * c.x;
        const uint32_t hi1 = __umulhi(kMul1, c.z), lo1 = kMul1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += kWeyl0;
        k.y += kWeyl1;
    }
    return c;
}

__device__ __forceinline__ double uniform53(uint32_t lo, uint32_t hi) {
    const uint64_t a = ((static_cast<uint64_t>(hi) << 32) | lo) >> 11;
    return (static_cast<double>(a) + 0.5) * 0x1.0p-53;
}

__global__ void k_philox_fields(double* __restrict__ out, uint2 key, uint32_t sys, int k0, int n, int W, int na) {
    const int npair = na / 2;
    const long total = (long)n * W * npair;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int j = (int)(t % npair);
        const long sw = t / npair;
        const int w = (int)(sw % W);
        const int s = (int)(sw / W);
        const uint4 r = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(k0 + s), (uint32_t)w, sys), key);
        const double u1 = uniform53(r.x, r.y), u2 = uniform53(r.z, r.w);
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincos(kTwoPi * u2, &sn, &cs);
        double* o = out + ((long)s * W + w) * na + 2 * j;
        o[0] = rad * cs;
        o[1] = rad * sn;
    }
}

}  // namespace

cudaError_t launch_philox_fields(double* out, uint64_t seed, uint32_t sys, int k0, int n, int W, int na,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long total = (long)n * W * (na / 2);
    const int threads = 256;
    const long blocks = std::min<long>((total + threads - 1) / threads, 152L * 32);
    const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    k_philox_fields<<<(unsigned)blocks, threads, 0, st>>>(out, key, sys, k0, n, W, na);
    return cudaGetLastError();
}

}  // namespace ftq

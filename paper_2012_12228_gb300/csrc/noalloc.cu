// Allocation-free estimator entry point.
//
// Some callers cannot let a library call cudaMalloc: applications whose
// device memory is owned by a framework's pool allocator under a fixed
// budget (a library-side cudaMalloc would bypass the pool and can fail or
// fragment it), and latency-sensitive loops that must not trigger the
// implicit device-wide synchronisation a cudaMalloc / cudaFree pair can
// cause.  For them ftq_estimators_noalloc evaluates the UEG estimators from
// a Green's function the caller already holds, with every piece of working
// memory (the momentum-transfer tables) in one file-scope device array of
// fixed size instead of a context.
#include <cmath>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "complex_math.cuh"
#include "ftq_internal.h"

namespace ftq {
void set_global_error(const std::string& msg);

namespace {

// Working memory of ftq_estimators_noalloc.  It lives as long as the
// library is loaded, on every device that runs the entry point.
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, fetched once
// per device (this is the call's only set-up work).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double2 p_elem(const double2* Gw, int M, int a, int b) {
    double2 g = Gw[(long)b * M + a];
    return make_double2((a == b ? 1.0 : 0.0) - g.x, -g.y);
}

__device__ double2 sum_block(double2 v, double2* sh) {
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_down(v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 acc = sh[0];
        for (int i = 1; i < (int)((blockDim.x + 31) >> 5); ++i) acc = acc + sh[i];
        sh[0] = acc;
    }
    __syncthreads();
    double2 r = sh[0];
    __syncthreads();
    return r;
}

// Same estimator algebra as the context path (P = I - G^T; N, E_1, Gamma,
// Lambda), tables read from the scratch array.
__global__ void k_estimators_noalloc(const double2* __restrict__ G, double* __restrict__ out,
                                     const int* __restrict__ pptr, const int* __restrict__ pa,
                                     const int* __restrict__ pb, const uint16_t* __restrict__ vidx,
                                     const double* __restrict__ vq, const double* __restrict__ ksq, int M, int nqh,
                                     double E_M) {
    extern __shared__ unsigned char smem_raw[];
    double2* rho = reinterpret_cast<double2*>(smem_raw);
    __shared__ double2 shc[32];
    const int w = blockIdx.x;
    const double2* Gw = G + (long)w * M * M;
    const int nt = blockDim.x;
    const int nslot = 2 * nqh + 1;
    for (int sl = 1 + threadIdx.x; sl < nslot; sl += nt) {
        double2 r = make_double2(0.0, 0.0);
        for (int e = pptr[sl]; e < pptr[sl + 1]; ++e) r = r + p_elem(Gw, M, pa[e], pb[e]);
        rho[sl] = r;
    }
    __syncthreads();
    double2 nsum = make_double2(0.0, 0.0), e1 = nsum, e2 = nsum;
    for (int a = threadIdx.x; a < M; a += nt) {
        double2 p = p_elem(Gw, M, a, a);
        nsum = nsum + p * 2.0;
        e1 = e1 + p * ksq[a];
    }
    for (int q = threadIdx.x; q < nqh; q += nt) e2 = e2 + cmul(rho[1 + 2 * q], rho[2 + 2 * q]) * (4.0 * vq[q]);
    const int npair = pptr[nslot];
    for (int e = threadIdx.x; e < npair; e += nt) {
        const int a = pa[e], d = pb[e];
        const int sl = vidx[(long)a * M + d];
        double2 lam = make_double2(0.0, 0.0);
        for (int f = pptr[sl]; f < pptr[sl + 1]; ++f) lam = cfma(p_elem(Gw, M, a, pa[f]), p_elem(Gw, M, pb[f], d), lam);
        e2 = e2 - lam * vq[(sl - 1) >> 1];
    }
    nsum = sum_block(nsum, shc);
    e1 = sum_block(e1, shc);
    e2 = sum_block(e2, shc);
    if (threadIdx.x == 0) {
        double* o = out + 8L * w;
        o[0] = 0.0; o[1] = 0.0; o[2] = 1.0;
        o[3] = E_M + e1.x + e2.x; o[4] = e1.y + e2.y;
        o[5] = nsum.x; o[6] = nsum.y; o[7] = 0.0;
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace
}  // namespace ftq

extern "C" int ftq_estimators_noalloc(int N, int M, double rs, const void* G_dev, int W, double* per_walker_dev,
                                      void* cuda_stream) {
    using namespace ftq;
    if (!G_dev || !per_walker_dev || W <= 0) {
        set_global_error("ftq_estimators_noalloc: NULL buffer or W <= 0");
        return FTQ_EINVAL;
    }
    if (N % 2 != 0) {
        set_global_error("ftq_estimators_noalloc: N must be even (unpolarised gas)");
        return FTQ_EINVAL;
    }
    UegSetup s;
    // theta and dtau do not enter the estimators; any positive values do
    std::string why = build_ueg(s, N, M, rs, 1.0, std::nan(""), 1.0);
    if (!why.empty()) {
        set_global_error("ftq_estimators_noalloc: " + why);
        return FTQ_EINVAL;
    }
    const int nslot = 2 * s.nq_half + 1;
    const size_t npair = s.pair_a.size();
    // packed layout of the tables inside the scratch array
    size_t off_ptr = 0;
    size_t off_a = align_up(off_ptr + sizeof(int) * (nslot + 1), 256);
    size_t off_b = align_up(off_a + sizeof(int) * npair, 256);
    size_t off_vidx = align_up(off_b + sizeof(int) * npair, 256);
    size_t off_vq = align_up(off_vidx + sizeof(uint16_t) * (size_t)M * M, 256);
    size_t off_ksq = align_up(off_vq + sizeof(double) * s.nq_half, 256);
    size_t total = align_up(off_ksq + sizeof(double) * M, 256);
    if (total > kNoAllocScratchBytes) {
        set_global_error("ftq_estimators_noalloc: the tables for M=" + std::to_string(M) + " need " +
                         std::to_string(total) + " bytes; the fixed scratch holds " +
                         std::to_string(kNoAllocScratchBytes) + " (use a context for larger bases)");
        return FTQ_EINVAL;
    }
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data() + off_ptr, s.pair_ptr.data(), sizeof(int) * (nslot + 1));
    std::memcpy(host.data() + off_a, s.pair_a.data(), sizeof(int) * npair);
    std::memcpy(host.data() + off_b, s.pair_b.data(), sizeof(int) * npair);
    std::memcpy(host.data() + off_vidx, s.vidx.data(), sizeof(uint16_t) * (size_t)M * M);
    std::memcpy(host.data() + off_vq, s.vq.data(), sizeof(double) * s.nq_half);
    std::vector<double> ksq(M);
    for (int i = 0; i < M; ++i) ksq[i] = 2.0 * s.eps[i];
    std::memcpy(host.data() + off_ksq, ksq.data(), sizeof(double) * M);

    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        set_global_error(std::string("ftq_estimators_noalloc: scratch address: ") + cudaGetErrorString(e));
        return FTQ_ECUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    unsigned char* b = static_cast<unsigned char*>(base);
    // a pageable source: the copy is staged before this call returns, so the
    // host vector may go out of scope afterwards
    e = cudaMemcpyAsync(b, host.data(), total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        size_t sm = sizeof(double2) * nslot;
        if (sm > 48 * 1024)
            e = cudaFuncSetAttribute(k_estimators_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) {
            k_estimators_noalloc<<<W, 256, sm, st>>>(
                static_cast<const double2*>(G_dev), per_walker_dev, reinterpret_cast<const int*>(b + off_ptr),
                reinterpret_cast<const int*>(b + off_a), reinterpret_cast<const int*>(b + off_b),
                reinterpret_cast<const uint16_t*>(b + off_vidx), reinterpret_cast<const double*>(b + off_vq),
                reinterpret_cast<const double*>(b + off_ksq), M, s.nq_half, s.E_M);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("ftq_estimators_noalloc: ") + cudaGetErrorString(e));
        return FTQ_ECUDA;
    }
    return FTQ_OK;
}

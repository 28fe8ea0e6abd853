// Density correlation <rho(Q) rho(-Q)> of every walker and its weighted
// average: the numerator of the static structure factor
// S(Q) = <rho(Q) rho(-Q)> / N (Results, structure factor), from
// P = I - G^T by Wick's theorem: Gamma_Q - Lambda_Q + D_Q with
// Gamma_Q = (2 rho_Q)(2 rho_-Q), Lambda_Q = 2 sum_{K1 K2} P_{K1+Q,K2} P_{K2-Q,K1}
// (the exchange sum of the energy estimator) and
// D_Q = 2 sum_{K: K, K+Q in basis} P_{K+Q,K+Q}.
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"

namespace ftq {
namespace {

// P_ab = <a+_a a_b> = delta_ab - G_ba
__device__ __forceinline__ double2 pel_s(const double2* Gw, int M, int a, int b) {
    const double2 g = Gw[(long)b * M + a];
    return make_double2((a == b ? 1.0 : 0.0) - g.x, -g.y);
}

// One block per walker; slot sl (1 .. nslot-1) is the transfer of the pair
// lists (odd: +q of the half space, even: -q).
__global__ void k_structure(const double2* __restrict__ G, const int* __restrict__ pptr,
                            const int* __restrict__ pa, const int* __restrict__ pb,
                            const uint16_t* __restrict__ vidx, double2* __restrict__ out, int M, int nslot) {
    extern __shared__ unsigned char smem_raw[];
    double2* rho = reinterpret_cast<double2*>(smem_raw);    // [nslot]
    double2* acc = rho + nslot;                             // [nslot]: D_Q - Lambda_Q
    const int w = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const double2* Gw = G + (long)w * M * M;
    for (int sl = 1 + tid; sl < nslot; sl += nt) {
        double2 r = make_double2(0.0, 0.0), d = make_double2(0.0, 0.0);
        for (int e = pptr[sl]; e < pptr[sl + 1]; ++e) {
            r = r + pel_s(Gw, M, pa[e], pb[e]);
            d = d + pel_s(Gw, M, pa[e], pa[e]);
        }
        rho[sl] = r;
        acc[sl] = d * 2.0;
    }
    __syncthreads();
    const int npair = pptr[nslot];
    for (int e = tid; e < npair; e += nt) {
        const int a = pa[e], d = pb[e];
        const int sl = vidx[(long)a * M + d];
        double2 lam = make_double2(0.0, 0.0);
        for (int f = pptr[sl]; f < pptr[sl + 1]; ++f) lam = cfma(pel_s(Gw, M, a, pa[f]), pel_s(Gw, M, pb[f], d), lam);
        atomicAdd(&acc[sl].x, -2.0 * lam.x);
        atomicAdd(&acc[sl].y, -2.0 * lam.y);
    }
    __syncthreads();
    for (int sl = 1 + tid; sl < nslot; sl += nt) {
        const int partner = (sl & 1) ? sl + 1 : sl - 1;
        const double2 gam = cmul(rho[sl] * 2.0, rho[partner] * 2.0);
        out[(long)w * (nslot - 1) + sl - 1] = gam + acc[sl];
    }
}

// Weights w = exp(ln|w| - s) e^{i arg w} of the alive walkers (s = max ln|w|)
// and their sum; one block.
__global__ void k_struct_weights(const double* __restrict__ ws, double2* __restrict__ wr, double* __restrict__ out,
                                 int W) {
    __shared__ double shm[32];
    __shared__ double2 shc[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    double m = -INFINITY;
    for (int i = tid; i < W; i += nt) {
        const double* s = ws + (long)WSTRIDE * i;
        if (s[2] > 0.5 && isfinite(s[0]) && s[0] > m) m = s[0];
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) shm[tid >> 5] = m;
    __syncthreads();
    double ref = shm[0];
    for (int i = 1; i < (nt + 31) / 32; ++i) ref = fmax(ref, shm[i]);
    __syncthreads();
    double2 sum = make_double2(0.0, 0.0);
    double nal = 0.0;
    for (int i = tid; i < W; i += nt) {
        const double* s = ws + (long)WSTRIDE * i;
        double2 v = make_double2(0.0, 0.0);
        if (s[2] > 0.5 && isfinite(s[0])) {
            const double mag = exp(s[0] - ref);
            v = make_double2(mag * cos(s[1]), mag * sin(s[1]));
            nal += 1.0;
        }
        wr[i] = v;
        sum = sum + v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum.x += __shfl_down_sync(0xffffffffu, sum.x, o);
        sum.y += __shfl_down_sync(0xffffffffu, sum.y, o);
        nal += __shfl_down_sync(0xffffffffu, nal, o);
    }
    if ((tid & 31) == 0) {
        shc[tid >> 5] = sum;
        shm[tid >> 5] = nal;
    }
    __syncthreads();
    if (tid == 0) {
        double2 t = shc[0];
        double n = shm[0];
        for (int i = 1; i < (nt + 31) / 32; ++i) {
            t = t + shc[i];
            n += shm[i];
        }
        out[0] = t.x;
        out[1] = t.y;
        out[2] = ref;
        out[3] = n;
    }
}

// sum_w w <rho(Q) rho(-Q)>_w for every slot (thread per slot).
__global__ void k_struct_reduce(const double2* __restrict__ wr, const double2* __restrict__ pw,
                                double* __restrict__ out, int W, int nq) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int w = 0; w < W; ++w) acc = cfma(wr[w], pw[(long)w * nq + j], acc);
    out[4 + 2 * j] = acc.x;
    out[5 + 2 * j] = acc.y;
}

}  // namespace

cudaError_t launch_structure_factor(ftq_ctx* c, double* per_walker_out) {
    const int W = c->W, nslot = c->nslot, nq = nslot - 1;
    cudaError_t e = cudaSuccess;
    if (!c->sq_walker) {
        e = cudaMalloc(&c->sq_walker, sizeof(double2) * (size_t)W * nq);
        if (e == cudaSuccess) e = cudaMalloc(&c->sq_w, sizeof(double2) * (size_t)W);
        if (e == cudaSuccess) e = cudaMalloc(&c->sq_out, sizeof(double) * (4 + 2 * (size_t)nq));
        if (e != cudaSuccess) return e;
    }
    if (!c->g64_valid) {
        e = mixed_sync_g64(c);
        if (e != cudaSuccess) return e;
    }
    const size_t sm = 2 * sizeof(double2) * (size_t)nslot;
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(k_structure, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    {
        LaunchScope ls(c, FTQ_K_ESTIMATORS);
        k_structure<<<W, 256, sm, c->stream>>>(c->G, c->tab.pair_ptr, c->tab.pair_a, c->tab.pair_b, c->tab.vidx,
                                              c->sq_walker, c->M, nslot);
    }
    {
        LaunchScope ls(c, FTQ_K_ESTIMATORS);
        k_struct_weights<<<1, 256, 0, c->stream>>>(c->wstate, c->sq_w, c->sq_out, W);
    }
    {
        LaunchScope ls(c, FTQ_K_ESTIMATORS);
        k_struct_reduce<<<(nq + 127) / 128, 128, 0, c->stream>>>(c->sq_w, c->sq_walker, c->sq_out, W, nq);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && per_walker_out)
        e = cudaMemcpyAsync(per_walker_out, c->sq_walker, sizeof(double2) * (size_t)W * nq, cudaMemcpyDeviceToDevice,
                            c->stream);
    return e;
}

}  // namespace ftq

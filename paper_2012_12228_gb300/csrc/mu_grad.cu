// Derivative of the estimators with respect to the chemical potential mu at
// tau = beta, at fixed draws x and with the force bias held at its value on
// the path.
//
// Every B carries the scalar factor exp(dtau mu), so along the path
//   d ln det(I + A_k)/dmu = k dtau (M - tr G(tau_k))
// (accumulated slice by slice into d ln|w|/dmu by the Green's-function
// kernels: d ln S_k = 2 (t_k - t_{k-1}), phaseless weight d ln|I_k| +
// d log cos theta_k = Re d ln S_k - tan(theta_k) Im d ln S_k), and at tau = beta
//   dG/dmu = -beta (I - G) G,   dP/dmu = -dG^T.
// The local energy and particle number are differentiated along dP
// (E_1 and N linearly, Gamma_Q and Lambda_Q by the product rule), and
//   d<O>/dmu = <dO + O d ln w> - <O><d ln w>.
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"

namespace ftq {
namespace {

template <typename T>
__device__ T bsum(T v, T* sh) {
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

// H = G - G G for every walker (32 x 32 output tiles, k tile 16).
__global__ void __launch_bounds__(256) k_g_minus_g2(const double2* __restrict__ G, double2* __restrict__ H, int M,
                                                   int tiles) {
    __shared__ double2 As[16][33];
    __shared__ double2 Bs[16][33];
    const int w = blockIdx.y;
    const int r0 = (blockIdx.x / tiles) * 32, c0 = (blockIdx.x % tiles) * 32;
    const double2* Gw = G + (long)w * M * M;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double2 acc[2][2] = {};
    for (int k0 = 0; k0 < M; k0 += 16) {
        for (int l = 0; l < 2; ++l) {
            const int e = threadIdx.x + 256 * l;
            const int r = e >> 4, kk = e & 15;
            As[kk][r] = (r0 + r < M && k0 + kk < M) ? Gw[(long)(r0 + r) * M + k0 + kk] : make_double2(0.0, 0.0);
            const int kb = e >> 5, cb = e & 31;
            Bs[kb][cb] = (k0 + kb < M && c0 + cb < M) ? Gw[(long)(k0 + kb) * M + c0 + cb] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const double2 a0 = As[kk][ty], a1 = As[kk][ty + 16], b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = cfma(a0, b0, acc[0][0]);
            acc[0][1] = cfma(a0, b1, acc[0][1]);
            acc[1][0] = cfma(a1, b0, acc[1][0]);
            acc[1][1] = cfma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int i = r0 + ty + 16 * a, c = c0 + tx + 16 * b;
            if (i < M && c < M) {
                const long e = (long)w * M * M + (long)i * M + c;
                H[e] = G[e] - acc[a][b];
            }
        }
}

__device__ __forceinline__ double2 p_of(const double2* Gw, int M, int a, int b) {
    const double2 g = Gw[(long)b * M + a];
    return make_double2((a == b ? 1.0 : 0.0) - g.x, -g.y);
}

__device__ __forceinline__ double2 dp_of(const double2* Hw, int M, int a, int b, double beta) {
    return Hw[(long)b * M + a] * beta;   // dP_ab = -dG_ba = beta H_ba
}

__global__ void k_est_dmu(const double2* __restrict__ G, const double2* __restrict__ H, const double* __restrict__ ws,
                          double* __restrict__ est, const int* __restrict__ pptr, const int* __restrict__ pa,
                          const int* __restrict__ pb, const uint16_t* __restrict__ vidx,
                          const double* __restrict__ vq, const double* __restrict__ ksq, int M, int nqh, double E_M,
                          double beta) {
    extern __shared__ unsigned char smem_raw[];
    const int nslot = 2 * nqh + 1;
    double2* rho = reinterpret_cast<double2*>(smem_raw);
    double2* drho = rho + nslot;
    __shared__ double2 shc[32];
    const int w = blockIdx.x, nt = blockDim.x;
    const double2* Gw = G + (long)w * M * M;
    const double2* Hw = H + (long)w * M * M;
    for (int sl = 1 + threadIdx.x; sl < nslot; sl += nt) {
        double2 r = make_double2(0.0, 0.0), dr = r;
        for (int e = pptr[sl]; e < pptr[sl + 1]; ++e) {
            r = r + p_of(Gw, M, pa[e], pb[e]);
            dr = dr + dp_of(Hw, M, pa[e], pb[e], beta);
        }
        rho[sl] = r;
        drho[sl] = dr;
    }
    __syncthreads();
    double2 n = make_double2(0.0, 0.0), dn = n, e1 = n, de1 = n, e2 = n, de2 = n;
    for (int a = threadIdx.x; a < M; a += nt) {
        const double2 p = p_of(Gw, M, a, a), dp = dp_of(Hw, M, a, a, beta);
        n = n + p * 2.0;
        dn = dn + dp * 2.0;
        e1 = e1 + p * ksq[a];
        de1 = de1 + dp * ksq[a];
    }
    for (int q = threadIdx.x; q < nqh; q += nt) {
        const double2 rp = rho[1 + 2 * q], rm = rho[2 + 2 * q];
        e2 = e2 + cmul(rp, rm) * (4.0 * vq[q]);
        de2 = de2 + (cmul(drho[1 + 2 * q], rm) + cmul(rp, drho[2 + 2 * q])) * (4.0 * vq[q]);
    }
    const int npair = pptr[nslot];
    for (int e = threadIdx.x; e < npair; e += nt) {
        const int a = pa[e], d = pb[e];
        const int sl = vidx[(long)a * M + d];
        double2 lam = make_double2(0.0, 0.0), dlam = lam;
        for (int f = pptr[sl]; f < pptr[sl + 1]; ++f) {
            const double2 pab = p_of(Gw, M, a, pa[f]), pcd = p_of(Gw, M, pb[f], d);
            lam = cfma(pab, pcd, lam);
            dlam = cfma(dp_of(Hw, M, a, pa[f], beta), pcd, cfma(pab, dp_of(Hw, M, pb[f], d, beta), dlam));
        }
        const double v = vq[(sl - 1) >> 1];
        e2 = e2 - lam * v;
        de2 = de2 - dlam * v;
    }
    n = bsum(n, shc);
    dn = bsum(dn, shc);
    e1 = bsum(e1, shc);
    de1 = bsum(de1, shc);
    e2 = bsum(e2, shc);
    de2 = bsum(de2, shc);
    if (threadIdx.x == 0) {
        const double* s = ws + (long)WSTRIDE * w;
        double* o = est + (long)WSTRIDE * w;
        o[0] = s[0]; o[1] = s[1]; o[2] = s[2];
        o[3] = E_M + e1.x + e2.x; o[4] = e1.y + e2.y;
        o[5] = n.x; o[6] = n.y; o[7] = 0.0;
        o[8] = s[8]; o[9] = s[11];
        o[10] = de1.x + de2.x; o[11] = de1.y + de2.y;
        o[12] = dn.x; o[13] = dn.y;
        o[14] = 0.0; o[15] = 0.0;
    }
}

// d<O>/dmu = sum w (dO + O dlnw) / sum w - <O> sum w dlnw / sum w over live walkers
__global__ void k_reduce_dmu(const double* __restrict__ est, double* __restrict__ out, int W) {
    __shared__ double2 shc[32];
    __shared__ double shm[32];
    __shared__ int shi[32];
    double best = -INFINITY;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const double* o = est + (long)WSTRIDE * w;
        if (o[2] > 0.5 && isfinite(o[0]) && o[0] > best) best = o[0];
    }
    for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = shm[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) b = fmax(b, shm[i]);
        shm[0] = b;
    }
    __syncthreads();
    const double s = isfinite(shm[0]) ? shm[0] : 0.0;
    double2 s0 = make_double2(0.0, 0.0), sE = s0, sN = s0, sd = s0, sdE = s0, sdN = s0;
    int nal = 0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const double* o = est + (long)WSTRIDE * w;
        if (o[2] <= 0.5 || !isfinite(o[0])) continue;     // a non-finite ln|w| weighs 0
        const double m = exp(o[0] - s);
        const double2 ww = make_double2(m * cos(o[1]), m * sin(o[1]));
        const double2 E = make_double2(o[3], o[4]), Nn = make_double2(o[5], o[6]);
        const double2 dl = make_double2(o[8], o[9]);
        const double2 dE = make_double2(o[10], o[11]), dN = make_double2(o[12], o[13]);
        s0 = s0 + ww;
        sE = sE + cmul(ww, E);
        sN = sN + cmul(ww, Nn);
        sd = sd + cmul(ww, dl);
        sdE = sdE + cmul(ww, dE + cmul(E, dl));
        sdN = sdN + cmul(ww, dN + cmul(Nn, dl));
        ++nal;
    }
    s0 = bsum(s0, shc);
    sE = bsum(sE, shc);
    sN = bsum(sN, shc);
    sd = bsum(sd, shc);
    sdE = bsum(sdE, shc);
    sdN = bsum(sdN, shc);
    for (int off = 16; off > 0; off >>= 1) nal += __shfl_down_sync(0xffffffffu, nal, off);
    if ((threadIdx.x & 31) == 0) shi[threadIdx.x >> 5] = nal;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += shi[i];
        const double2 inv = cinv(s0);
        const double2 mE = cmul(sE, inv), mN = cmul(sN, inv), md = cmul(sd, inv);
        const double2 dE = cmul(sdE, inv) - cmul(mE, md);
        const double2 dN = cmul(sdN, inv) - cmul(mN, md);
        out[0] = dN.x; out[1] = dE.x; out[2] = mN.x; out[3] = mE.x;
        out[4] = (double)tot; out[5] = s; out[6] = dN.y; out[7] = dE.y;
    }
}

}  // namespace

cudaError_t launch_mu_grad(ftq_ctx* c, double* per_walker) {
    const int M = c->M, nqh = c->sys.nq_half;
    if (!c->g64_valid) {
        cudaError_t e0 = mixed_sync_g64(c);
        if (e0 != cudaSuccess) return e0;
    }
    const int tiles = (M + 31) / 32;
    {
        LaunchScope ls(c, FTQ_K_ESTIMATORS);
        k_g_minus_g2<<<dim3((unsigned)(tiles * tiles), (unsigned)c->W), 256, 0, c->stream>>>(c->G, c->work, M, tiles);
    }
    const size_t sm = 2 * sizeof(double2) * (2 * nqh + 1);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_est_dmu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    {
        LaunchScope ls(c, FTQ_K_ESTIMATORS);
        k_est_dmu<<<c->W, 256, sm, c->stream>>>(c->G, c->work, c->wstate, c->est, c->tab.pair_ptr, c->tab.pair_a,
                                                c->tab.pair_b, c->tab.vidx, c->tab.vq, c->tab.ksq, M, nqh, c->sys.E_M,
                                                c->sys.beta);
    }
    {
        LaunchScope ls(c, FTQ_K_ESTIMATORS);
        k_reduce_dmu<<<1, 256, 0, c->stream>>>(c->est, c->red + 8, c->W);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (per_walker)
        e = cudaMemcpy2DAsync(per_walker, sizeof(double) * 8, c->est + 8, sizeof(double) * WSTRIDE,
                              sizeof(double) * 8, c->W, cudaMemcpyDeviceToDevice, c->stream);
    return e;
}

}  // namespace ftq

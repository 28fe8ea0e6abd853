// UEG estimators (Sec. "Uniform Electron Gas", local energy; Results, the
// time-slice estimates and their average).
//
// Per walker, from P = I - G^T:
//   N = 2 tr P,  E_1 = sum_K |K|^2 P_KK,  rho_Q = sum_{K} P_{K+Q,K},
//   E_2 = sum_q 4 v_q rho_q rho_-q - sum_Q v_Q Lambda_Q,
//   Lambda_Q = sum over the pairs (a, d), (b, c) of transfer Q of P_ab P_cd.
// Lambda_-Q = Lambda_Q (the pairs of -Q are those of +Q reversed, and the sum
// is the trace of a product of two gathered blocks, tr(XY) = tr(YX)), so only
// the half-space transfers are summed and counted twice.
//
// k_est_walkers: persistent blocks over walkers (a walker's G stays in L2
// while its block works on it); a warp per slot for rho, a warp per +Q pair
// (a, d) for Lambda with lanes over the pairs of the same transfer.  Each
// lane scales its partial sum by v_Q and keeps it, so no reduction is needed
// per pair.  T = double2 reads a complex128 G and sums in FP64; T = float2
// reads the FP32 G of the mixed path's slices, forms the products and the
// per-pair partial sums in FP32 and accumulates them in FP64.
#include <cmath>

#include "block_reduce.cuh"
#include "complex_math.cuh"
#include "ftq_internal.h"

namespace ftq {
namespace {

__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }

// P_ab = delta_ab - G_ba in the arithmetic of T
__device__ __forceinline__ double2 pel(const double2* Gw, int M, int a, int b) {
    const double2 g = Gw[(long)b * M + a];
    return make_double2((a == b ? 1.0 : 0.0) - g.x, -g.y);
}
__device__ __forceinline__ float2 pel(const float2* Gw, int M, int a, int b) {
    const float2 g = Gw[(long)b * M + a];
    return make_float2((a == b ? 1.f : 0.f) - g.x, -g.y);
}

__device__ __forceinline__ double2 warp_sum_d(double2 v) {
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_down(v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(512) k_est_walkers(const T* __restrict__ G, const double* __restrict__ ws,
                                                    double* __restrict__ est, const int* __restrict__ pptr,
                                                    const int* __restrict__ pa, const int* __restrict__ pb,
                                                    const uint16_t* __restrict__ vidx, const int* __restrict__ eplus,
                                                    int neplus, const double* __restrict__ vq,
                                                    const double* __restrict__ ksq, int M, int nqh, double E_M,
                                                    int W) {
    extern __shared__ unsigned char smem_raw[];
    double2* rho = reinterpret_cast<double2*>(smem_raw);     // [2 nqh + 1]
    __shared__ double2 shc[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nslot = 2 * nqh + 1;
    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        const T* Gw = G + (size_t)w * M * M;
        for (int sl = 1 + warp; sl < nslot; sl += nw) {
            double2 r = make_double2(0.0, 0.0);
            for (int e = pptr[sl] + lane; e < pptr[sl + 1]; e += 32) r = r + to_d(pel(Gw, M, pa[e], pb[e]));
            r = warp_sum_d(r);
            if (lane == 0) rho[sl] = r;
        }
        __syncthreads();
        double2 nsum = make_double2(0.0, 0.0), e1 = nsum, e2 = nsum, ex = nsum;
        for (int a = threadIdx.x; a < M; a += blockDim.x) {
            const double2 p = to_d(pel(Gw, M, a, a));
            nsum = nsum + p * 2.0;
            e1 = e1 + p * ksq[a];
        }
        for (int q = threadIdx.x; q < nqh; q += blockDim.x) e2 = e2 + cmul(rho[1 + 2 * q], rho[2 + 2 * q]) * (4.0 * vq[q]);
        for (int t = warp; t < neplus; t += nw) {
            const int e = eplus[t];
            const int a = pa[e], d = pb[e];
            const int sl = vidx[(long)a * M + d];
            T acc;
            acc.x = 0;
            acc.y = 0;
            for (int f = pptr[sl] + lane; f < pptr[sl + 1]; f += 32)
                acc = cfma(pel(Gw, M, a, pa[f]), pel(Gw, M, pb[f], d), acc);
            ex = ex + to_d(acc) * vq[(sl - 1) >> 1];
        }
        e2 = e2 - ex * 2.0;
        nsum = block_sum(nsum, shc);
        e1 = block_sum(e1, shc);
        e2 = block_sum(e2, shc);
        if (threadIdx.x == 0) {
            const double* s = ws + (long)WSTRIDE * w;
            double* o = est + (long)WSTRIDE * w;
            o[0] = s[0]; o[1] = s[1]; o[2] = s[2];
            o[3] = E_M + e1.x + e2.x; o[4] = e1.y + e2.y;
            o[5] = nsum.x; o[6] = nsum.y; o[7] = 0.0;
        }
    }
}

// sum_w of w, wE, wN with w = exp(ln|w| - s) e^{i arg w}, s = max ln|w| over
// the alive walkers with a finite ln|w| (the others weigh 0); writes
// {Re, Im sum w, Re, Im sum wE, Re, Im sum wN, s, alive} to out, and when
// rec is given also {k, E_k, N_k, alive, Re sum w, s} to rec.
__global__ void k_reduce_walkers(const double* __restrict__ est, double* __restrict__ out, int W,
                                 double* __restrict__ rec, int k) {
    __shared__ double shv[32];
    __shared__ int shi[32];
    __shared__ double2 shc[32];
    double best = -INFINITY;
    int bi = W;
    for (int w = threadIdx.x; w < W; w += blockDim.x)
        if (est[(long)WSTRIDE * w + 2] > 0.5 && isfinite(est[(long)WSTRIDE * w]) && est[(long)WSTRIDE * w] > best) {
            best = est[(long)WSTRIDE * w];
            bi = w;
        }
    int wm = block_argmax(best, bi, shv, shi);
    double s = wm < W ? est[(long)WSTRIDE * wm] : 0.0;
    double2 sw = make_double2(0.0, 0.0), swe = sw, swn = sw;
    double nal = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const double* o = est + (long)WSTRIDE * w;
        if (o[2] <= 0.5 || !isfinite(o[0])) continue;     // a non-finite ln|w| weighs 0
        double m = exp(o[0] - s);
        double2 ww = make_double2(m * cos(o[1]), m * sin(o[1]));
        sw = sw + ww;
        swe = swe + cmul(ww, make_double2(o[3], o[4]));
        swn = swn + cmul(ww, make_double2(o[5], o[6]));
        nal += 1.0;
    }
    sw = block_sum(sw, shc);
    swe = block_sum(swe, shc);
    swn = block_sum(swn, shc);
    nal = block_sum(nal, shv);
    if (threadIdx.x == 0) {
        out[0] = sw.x; out[1] = sw.y; out[2] = swe.x; out[3] = swe.y;
        out[4] = swn.x; out[5] = swn.y; out[6] = s; out[7] = nal;
        if (rec) {
            const double2 E = nal > 0.0 ? cdiv(swe, sw) : make_double2(NAN, NAN);
            const double2 N = nal > 0.0 ? cdiv(swn, sw) : make_double2(NAN, NAN);
            rec[0] = (double)k; rec[1] = E.x; rec[2] = E.y; rec[3] = N.x; rec[4] = N.y;
            rec[5] = nal; rec[6] = sw.x; rec[7] = s;
        }
    }
}

// Row 0 of the slice summary: the number of recorded slices and the averages
// of their global estimates (each slice counts once); rows 1.. the records.
__global__ void k_slice_summary(const double* __restrict__ rec, int n, double* __restrict__ out, int rows) {
    __shared__ double2 shc[32];
    double2 e = make_double2(0.0, 0.0), nn = e;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        e = e + make_double2(rec[8 * r + 1], rec[8 * r + 2]);
        nn = nn + make_double2(rec[8 * r + 3], rec[8 * r + 4]);
    }
    e = block_sum(e, shc);
    nn = block_sum(nn, shc);
    if (threadIdx.x == 0) {
        const double inv = n > 0 ? 1.0 / n : NAN;
        out[0] = (double)n;
        out[1] = e.x * inv; out[2] = e.y * inv; out[3] = nn.x * inv; out[4] = nn.y * inv;
        out[5] = out[6] = out[7] = 0.0;
    }
    for (int i = threadIdx.x; i < 8 * rows; i += blockDim.x) out[8 + i] = rec[i];
}

template <typename T>
cudaError_t launch_est_walkers(ftq_ctx* c, const T* G) {
    const int nqh = c->sys.nq_half;
    const size_t sm = sizeof(double2) * (2 * nqh + 1);
    static size_t sm_set[2] = {48 * 1024, 48 * 1024};
    const int which = sizeof(T) == sizeof(double2) ? 0 : 1;
    if (sm > sm_set[which]) {
        cudaError_t e = cudaFuncSetAttribute(k_est_walkers<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        sm_set[which] = sm;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = c->W < 2 * sms ? c->W : 2 * sms;
    LaunchScope ls(c, FTQ_K_ESTIMATORS);
    k_est_walkers<T><<<grid, 512, sm, c->stream>>>(G, c->wstate, c->est, c->tab.pair_ptr, c->tab.pair_a,
                                                   c->tab.pair_b, c->tab.vidx, c->tab.eplus, c->tab.neplus,
                                                   c->tab.vq, c->tab.ksq, c->M, nqh, c->sys.E_M, c->W);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_estimators(ftq_ctx* c, double* per_walker) {
    if (!c->g64_valid) {
        cudaError_t e0 = mixed_sync_g64(c);
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = launch_est_walkers(c, c->G);
    if (e != cudaSuccess) return e;
    c->launches[FTQ_K_ESTIMATORS] += 1;
    k_reduce_walkers<<<1, 256, 0, c->stream>>>(c->est, c->red, c->W, nullptr, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (per_walker)
        e = cudaMemcpy2DAsync(per_walker, sizeof(double) * 8, c->est, sizeof(double) * WSTRIDE, sizeof(double) * 8,
                              c->W, cudaMemcpyDeviceToDevice, c->stream);
    return e;
}

cudaError_t launch_slice_estimate(ftq_ctx* c, int k) {
    if (c->trk_n >= c->sys.n_slices) return cudaErrorInvalidValue;
    // the mixed path holds G(tau_k) in FP32 for k < n and in complex128 at tau = beta
    cudaError_t e = c->g64_valid ? launch_est_walkers(c, c->G) : launch_est_walkers(c, c->G32);
    if (e != cudaSuccess) return e;
    c->launches[FTQ_K_ESTIMATORS] += 1;
    k_reduce_walkers<<<1, 256, 0, c->stream>>>(c->est, c->red, c->W, c->trk + 8 * (size_t)c->trk_n, k);
    c->trk_n += 1;
    return cudaGetLastError();
}

cudaError_t launch_slice_summary(ftq_ctx* c, double* out_dev, int rows) {
    k_slice_summary<<<1, 256, 0, c->stream>>>(c->trk, c->trk_n, out_dev, rows);
    c->launches[FTQ_K_ESTIMATORS] += 1;
    return cudaGetLastError();
}

}  // namespace ftq

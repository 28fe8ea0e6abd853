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
// while its block works on it); a warp per slot for rho; for Lambda a warp
// per work unit = 32 consecutive pairs (a, d) of one +Q transfer (one per
// lane), looping over all pairs (b, c) of that transfer: P_ab = delta_ab -
// G[b][a] is read from row b of G and P_cd = delta_cd - G[d][c] from row c
// of G^T (written by k_transpose_g), so the 32 lanes of a load touch
// neighbouring columns of one row, which needs few sectors.  With FP32 G
// each lane accumulates v_Q times its partial sum as a compensated float
// pair (two-sum), so no FP64 instruction runs per unit; with complex128 G the
// products and sums are FP64 (the FP64 pipe bounds that variant).
// T = double2 reads a complex128 G; T = float2 the FP32 G of the mixed
// path's slices.
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

// The delta terms of (delta_1 - g1)(delta_2 - g2) - g1 g2.
__device__ __forceinline__ double2 delta_terms(bool d1, bool d2, double2 g1, double2 g2) {
    double2 r = make_double2((d1 && d2) ? 1.0 : 0.0, 0.0);
    if (d1) r = r - g2;
    if (d2) r = r - g1;
    return r;
}
__device__ __forceinline__ float2 delta_terms(bool d1, bool d2, float2 g1, float2 g2) {
    float2 r = make_float2((d1 && d2) ? 1.f : 0.f, 0.f);
    if (d1) r = r - g2;
    if (d2) r = r - g1;
    return r;
}

// Gt[w] = G[w]^T through 32 x 33 shared tiles; grid (tiles, tiles, W).
template <typename T>
__global__ void k_transpose_g(const T* __restrict__ G, T* __restrict__ Gt, int M) {
    __shared__ T tile[32][33];
    const size_t off = (size_t)blockIdx.z * M * M;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = r0 + r, j = c0 + threadIdx.x;
        if (i < M && j < M) tile[r][threadIdx.x] = G[off + (size_t)i * M + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = c0 + r, i = r0 + threadIdx.x;
        if (i < M && j < M) Gt[off + (size_t)j * M + i] = tile[threadIdx.x][r];
    }
}

__device__ __forceinline__ double2 warp_sum_d(double2 v) {
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_down(v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_est_walkers(const T* __restrict__ G, const T* __restrict__ Gtr,
                                                     const double* __restrict__ ws,
                                                    double* __restrict__ est, const int* __restrict__ pptr,
                                                    const int* __restrict__ pa, const int* __restrict__ pb,
                                                    const uint16_t* __restrict__ vidx, const int4* __restrict__ units,
                                                    int nunits, const double* __restrict__ vq,
                                                    const float2* __restrict__ vqf,
                                                    const double* __restrict__ ksq, int M, int nqh, double E_M,
                                                    int W) {
    extern __shared__ unsigned char smem_raw[];
    double2* rho = reinterpret_cast<double2*>(smem_raw);     // [2 nqh + 1]
    __shared__ double2 shc[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nslot = 2 * nqh + 1;
    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        const T* Gw = G + (size_t)w * M * M;
        const T* Gt = Gtr + (size_t)w * M * M;
        for (int sl = 1 + warp; sl < nslot; sl += nw) {
            double2 r = make_double2(0.0, 0.0);
            for (int e = pptr[sl] + lane; e < pptr[sl + 1]; e += 32) r = r + to_d(pel(Gw, M, pa[e], pb[e]));
            r = warp_sum_d(r);
            if (lane == 0) rho[sl] = r;
        }
        __syncthreads();
        double2 nsum = make_double2(0.0, 0.0), e1 = nsum, e2 = nsum, ex = nsum;
        // FP32 G: v_Q acc accumulated per lane as a compensated float sum
        // (hi + lo, two-sum), so that no FP64 instruction runs per pair
        float exh[2] = {0.f, 0.f}, exl[2] = {0.f, 0.f};
        for (int a = threadIdx.x; a < M; a += blockDim.x) {
            const double2 p = to_d(pel(Gw, M, a, a));
            nsum = nsum + p * 2.0;
            e1 = e1 + p * ksq[a];
        }
        for (int q = threadIdx.x; q < nqh; q += blockDim.x) e2 = e2 + cmul(rho[1 + 2 * q], rho[2 + 2 * q]) * (4.0 * vq[q]);
        for (int u = warp; u < nunits; u += nw) {
            const int4 un = units[u];                  // slot pairs [x, y), chunk from z, v_Q index w
            const int f = un.z + lane;
            const bool on = f < un.y;
            const int al = on ? pa[f] : 0, dl = on ? pb[f] : 0;
            const T* gcol = Gw + al;                   // G[b][al] = gcol[b * M]
            const T* tcol = Gt + dl;                   // G[dl][c] = G^T[c][dl] = tcol[c * M]
            // P_ab P_cd = (delta_ab - g1)(delta_cd - g2) with g1 = G[b][a],
            // g2 = G[d][c]: the product g1 g2 every time, the delta terms
            // only where an index matches (once per lane and unit at most)
            T acc, acc2;
            acc.x = 0;
            acc.y = 0;
            acc2 = acc;
            int g = un.x;
#pragma unroll 1
            for (; g + 1 < un.y; g += 2) {
                const int b0 = pa[g], c0 = pb[g], b1 = pa[g + 1], c1 = pb[g + 1];   // the same for every lane
                const T x0 = gcol[(size_t)b0 * M], y0 = tcol[(size_t)c0 * M];
                const T x1 = gcol[(size_t)b1 * M], y1 = tcol[(size_t)c1 * M];
                acc = cfma(x0, y0, acc);
                acc2 = cfma(x1, y1, acc2);
                if (al == b0 || c0 == dl) acc = acc + delta_terms(al == b0, c0 == dl, x0, y0);
                if (al == b1 || c1 == dl) acc2 = acc2 + delta_terms(al == b1, c1 == dl, x1, y1);
            }
            if (g < un.y) {
                const int b0 = pa[g], c0 = pb[g];
                const T x0 = gcol[(size_t)b0 * M], y0 = tcol[(size_t)c0 * M];
                acc = cfma(x0, y0, acc);
                if (al == b0 || c0 == dl) acc = acc + delta_terms(al == b0, c0 == dl, x0, y0);
            }
            acc = acc + acc2;
            if (!on) continue;
            const int qi = un.w;
            if constexpr (sizeof(T) == sizeof(float2)) {
                const float2 v = vqf[qi];
                const float av[2] = {(float)acc.x, (float)acc.y};
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float pp = av[r] * v.x;
                    float ee = fmaf(av[r], v.x, -pp);
                    ee = fmaf(av[r], v.y, ee);
                    const float sum = exh[r] + pp;
                    const float bb = sum - exh[r];
                    exl[r] += ((exh[r] - (sum - bb)) + (pp - bb)) + ee;
                    exh[r] = sum;
                }
            } else {
                ex = ex + to_d(acc) * vq[qi];
            }
        }
        if constexpr (sizeof(T) == sizeof(float2))
            ex = make_double2((double)exh[0] + (double)exl[0], (double)exh[1] + (double)exl[1]);
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
    const int M = c->M;
    const size_t sm = sizeof(double2) * (2 * nqh + 1);
    if (sm > 220 * 1024) return cudaErrorInvalidValue;      // the transfer table alone is too large
    static size_t sm_set[2] = {48 * 1024, 48 * 1024};
    const bool f32 = sizeof(T) == sizeof(float2);
    const int which = f32 ? 1 : 0;
    if (sm > sm_set[which]) {
        cudaError_t e = cudaFuncSetAttribute(k_est_walkers<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        sm_set[which] = sm;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // FP32 G: one 1024-thread block per SM, so that fewer walkers compete for
    // the L2; complex128 G (FP64-pipe bound): two 512-thread blocks per SM
    const int nthr = f32 ? 1024 : 512;
    const int per_sm = f32 ? 1 : 2;
    const int grid = c->W < per_sm * sms ? c->W : per_sm * sms;
    LaunchScope ls(c, FTQ_K_ESTIMATORS);
    // G^T into the complex128 work buffer (scratch between calls; it holds a
    // complex128 or a complex64 matrix per walker)
    T* Gt = reinterpret_cast<T*>(c->work);
    const int tiles = (M + 31) / 32;
    k_transpose_g<T><<<dim3((unsigned)tiles, (unsigned)tiles, (unsigned)c->W), dim3(32, 8), 0, c->stream>>>(G, Gt, M);
    c->launches[FTQ_K_ESTIMATORS] += 1;
    k_est_walkers<T><<<grid, nthr, sm, c->stream>>>(G, Gt, c->wstate, c->est, c->tab.pair_ptr, c->tab.pair_a,
                                                    c->tab.pair_b, c->tab.vidx, c->tab.eplus, c->tab.neplus,
                                                    c->tab.vq, c->tab.vqf, c->tab.ksq, M, nqh, c->sys.E_M, c->W);
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

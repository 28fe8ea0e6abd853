// Green's function of the mixed path with the rank-16 updates on the tensor
// cores (tcgen05.mma kind::tf32, 3xTF32: hi*hi + hi*lo + lo*hi, FP32
// accumulation in TMEM).
//
// The algebra is that of the blocked LU kernel, G(tau) = I - B Mt^-1 D_Ls with
// Mt = D_Lb T^-1 D_Rb + D_Ls Y D_Rs and B = Y D_Rs (two-sided scale split of
// Q D T), but B Mt^-1 is formed by one Gauss-Jordan sweep instead of an LU and
// two triangular solves.  Per walker the kernel holds S = [Mt^T | B^T]
// (M rows, 2M columns; row r is [Re S[r][0..2M) | Im S[r][0..2M)], rows PL
// floats per part apart so that every 16-column chunk is 16-byte aligned)
// and reduces its left half to a permutation by row operations:
//
//   for each panel of 16 columns p..p+15:
//     1. partial pivoting on the panel (shared memory, CUDA cores): the
//        pivot rows pi_q are the rows an LU with partial pivoting would pick,
//        and the panel's pivot block factorises as P_pi = L_pi U_pi;
//     2. R = P_pi^-1 S[pi, c] for every column c right of the panel (one
//        column per thread), written into the pivot rows and, split into tf32
//        hi + lo, into the MMA's B operand;
//     3. S[r, c] -= P[r, :] R[:, c] for every other row r: a rank-16 update,
//        128 x N x 32 real-embedded MMAs (A rows [Re ; Im] of 64 complex rows,
//        A = [[Pr, -Pi], [Pi, Pr]] from the panel as it was before step 1).
//
// At the end the right half holds B Mt^-1 with its columns permuted:
// (B Mt^-1)[i][c] = S[pi_c][M + i].  det Mt is the product of the pivots
// times the sign of pi.  Gauss-Jordan takes 1.5 M^3 complex multiply-adds
// against 4/3 M^3 for LU and two solves; the tensor cores absorb the
// difference, and one uniform sweep keeps every update the same GEMM shape.
//
// One block of 256 threads per walker (two per SM at M = 257), S in the
// FP32 workspace (L2 / HBM).  Every wait on the MMA barrier is bounded: on
// expiry bit 2 of the status word is set, the block drains its MMAs
// (bounded), frees TMEM and returns without touching G or the weights.
#include <cmath>

#include "block_reduce.cuh"
#include "complex_math.cuh"
#include "ftq_internal.h"
#include "green_tail.cuh"
#include "mixed_common.cuh"
#include "tc_common.cuh"

namespace ftq {
namespace {

using namespace tc;

constexpr int GNB = 16;            // panel width: 16 complex columns = one 32-float operand row
constexpr int GTH = 256;           // threads per block
constexpr int ABYTES = 128 * 128;  // one tf32 part of the A operand: 128 rows x 32 floats
constexpr int TILE_BYTES = 32 * 33 * (int)sizeof(float2);
constexpr int NTMAX = 128;         // widest N tile: 2 warps per TMEM lane quarter x NCHW chunks of 16
constexpr int NCHW = NTMAX / 32;   // 16-column chunks per warp and tile

// Shared-memory layout (byte offsets from a 1024-aligned base) for basis size
// M and N tile NT.
struct GjLayout {
    size_t bhi, blo, pan, lupp, ipv, ppiv, drs, upiv, dls, dlb, drb, piv, pstep, total;
    __host__ __device__ GjLayout(int M, int NT) {
        bhi = 2 * (size_t)ABYTES;
        blo = bhi + (size_t)NT * 128;
        pan = blo + (size_t)NT * 128;
        size_t panb = (size_t)GNB * M * sizeof(float2);
        if (panb < (size_t)TILE_BYTES) panb = TILE_BYTES;
        lupp = pan + panb;
        ipv = lupp + GNB * GNB * sizeof(float2);
        ppiv = ipv + GNB * sizeof(float2);
        drs = ppiv + GNB * sizeof(int);
        upiv = drs + (size_t)M * sizeof(float2);
        dls = upiv + (size_t)M * sizeof(float2);
        dlb = dls + (size_t)M * sizeof(float);
        drb = dlb + (size_t)M * sizeof(float);
        piv = drb + (size_t)M * sizeof(float);
        pstep = piv + (size_t)M * sizeof(int);
        total = pstep + (size_t)M * sizeof(int) + 1024;   // + alignment slack
    }
};

__device__ __forceinline__ float2 csub_mul(float2 acc, float2 a, float2 b) {
    // acc - a * b
    return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}

// Block-wide argmax (ties to the lower index) with one barrier; every thread
// reduces the per-warp results itself.  Consecutive calls alternate between
// two buffers, so one barrier per call suffices.
__device__ __forceinline__ int gj_argmax(float val, int idx, float* shv, int* shi) {
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, val, o);
        const int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { shv[wid] = val; shi[wid] = idx; }
    __syncthreads();
    float bv = shv[0];
    int bi = shi[0];
#pragma unroll
    for (int i = 1; i < GTH / 32; ++i)
        if (shv[i] > bv || (shv[i] == bv && shi[i] < bi)) { bv = shv[i]; bi = shi[i]; }
    return bi;
}

// Floats per part (Re or Im) of a row of S: 2M rounded up to a multiple of 4,
// so that rows start on 16-byte boundaries.
__host__ __device__ __forceinline__ int gj_part_len(int M) { return (2 * M + 3) & ~3; }

__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float v) {
    float h, l;
    split_tf32(v, h, l);
    *reinterpret_cast<float*>(hi + off) = h;
    *reinterpret_cast<float*>(lo + off) = l;
}

__global__ void __launch_bounds__(GTH, 2) k_green_tc(const float* __restrict__ Ypl, const double2* __restrict__ Tinv,
                                                    const double2* __restrict__ DR, float2* __restrict__ work,
                                                    float2* __restrict__ G,
                                                    const double* __restrict__ eps, double* __restrict__ ws,
                                                    int* __restrict__ status, int M, double lscale, double mu_T,
                                                    int constraint, Planes P, size_t wstride, double kdt, int NT,
                                                    long long wait_limit) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_sh;
    __shared__ float shv[2][GTH / 32];
    __shared__ int shi[2][GTH / 32];
    __shared__ double shd[GTH / 32];
    __shared__ double2 shc[GTH / 32];
    __shared__ int nswap_sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    unsigned char* base = smem_raw + pad;
    const GjLayout L(M, NT);
    unsigned char* Ahi = base;
    unsigned char* Alo = base + ABYTES;
    unsigned char* Bhi = base + L.bhi;
    unsigned char* Blo = base + L.blo;
    float2* Pan = reinterpret_cast<float2*>(base + L.pan);      // [GNB][M] panel, column-major
    float2* LUpp = reinterpret_cast<float2*>(base + L.lupp);    // [GNB][GNB] pivot block: L below, U on and above
    float2* ipv = reinterpret_cast<float2*>(base + L.ipv);      // [GNB] inverse pivots of the panel
    int* ppiv = reinterpret_cast<int*>(base + L.ppiv);          // [GNB] pivot rows of the panel
    float2* drs = reinterpret_cast<float2*>(base + L.drs);      // [M]
    float2* upiv = reinterpret_cast<float2*>(base + L.upiv);    // [M] pivots in elimination order
    float* dls = reinterpret_cast<float*>(base + L.dls);        // [M]
    float* dlb = reinterpret_cast<float*>(base + L.dlb);        // [M]
    float* drb = reinterpret_cast<float*>(base + L.drb);        // [M]
    int* piv = reinterpret_cast<int*>(base + L.piv);            // [M] pivot row of elimination step s
    int* pstep = reinterpret_cast<int*>(base + L.pstep);        // [M] step at which row r was pivot (M: not yet)

    const int w = blockIdx.x;
    const int PL = gj_part_len(M);                              // floats per part of a row of S
    const size_t RS = 2 * (size_t)PL;                           // row stride of S (floats)
    float* Sw = reinterpret_cast<float*>(work) + (size_t)w * M * RS;
    // element (r, c) of S: Re at re(r, c), Im at re(r, c) + PL
    auto re = [&](int r, int c) -> float* { return Sw + (size_t)r * RS + c; };
    const float* Yw = Ypl + wstride * w;
    const double2* Tw = Tinv + (size_t)w * M * M;
    float2* Gw = G + (size_t)w * M * M;

    double lsum = 0.0;
    for (int i = tid; i < M; i += GTH) {
        const double dl = exp(-lscale * (eps[i] - mu_T));
        double b, s2;
        if (dl > 1.0) { b = 1.0 / dl; s2 = 1.0; } else { b = 1.0; s2 = dl; }
        dlb[i] = (float)b;
        dls[i] = (float)s2;
        const double2 d = DR[(long)w * M + i];
        const double a = sqrt(abs2(d));
        double rb;
        double2 rs;
        if (a > 1.0) { rb = 1.0 / a; rs = d * (1.0 / a); } else { rb = 1.0; rs = d; }
        drb[i] = (float)rb;
        drs[i] = make_float2((float)rs.x, (float)rs.y);
        lsum += log(b) + log(rb);
        pstep[i] = M;
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (wid == 0) tmem_alloc(&tmem_sh, (uint32_t)NT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;

    // ------------------------------------------------------------ build S
    // row j of S = [column j of Mt | column j of B].  The chain planes hold Y
    // by columns (contiguous over the row index n); T^-1 is row-major, so it
    // passes through 32 x 33 shared tiles.
    {
        float2* tile = Pan;
        for (int jb = 0; jb < M; jb += 32)
            for (int nb0 = 0; nb0 < M; nb0 += 32) {
                double2 tv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int n = nb0 + wid + 8 * u, j = jb + lane;
                    tv[u] = (n < M && j < M) ? Tw[(size_t)n * M + j] : make_double2(0.0, 0.0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int n = nb0 + wid + 8 * u, j = jb + lane;
                    const double sc = (n < M && j < M) ? (double)dlb[n] * (double)drb[j] : 0.0;
                    tile[(wid + 8 * u) * 33 + lane] = make_float2((float)(tv[u].x * sc), (float)(tv[u].y * sc));
                }
                __syncthreads();
                float2 yv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = jb + wid + 8 * u, n = nb0 + lane;
                    yv[u] = (n < M && j < M) ? P.load(Yw, n, j) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = wid + 8 * u, j = jb + r, n = nb0 + lane;
                    if (n < M && j < M) {
                        const float2 yd = cmul(yv[u], drs[j]);                     // B[n][j] = Y[n][j] D_Rs[j]
                        const float2 t = tile[lane * 33 + r];                      // D_Lb T^-1 D_Rb [n][j]
                        float* sj = re(j, 0);
                        sj[n] = t.x + yd.x * dls[n];                               // Mt[n][j]
                        sj[PL + n] = t.y + yd.y * dls[n];
                        sj[M + n] = yd.x;
                        sj[PL + M + n] = yd.y;
                    }
                }
                __syncthreads();
            }
    }

    // ------------------------------------------------------------ Gauss-Jordan sweep
    uint32_t phase = 0;
    int par = 0;
    bool aborted = false;
    for (int p = 0; p < M && !aborted; p += GNB) {
        const int nb = min(GNB, M - p);
        for (int e0 = 0; e0 < nb * M; e0 += 4 * GTH) {
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + tid + u * GTH;          // (row, column) with the column fastest
                v[u] = make_float2(0.f, 0.f);
                if (e < nb * M) {
                    const int r = e / nb, q = e - r * nb;
                    const float* a = re(r, p + q);
                    v[u] = make_float2(a[0], a[PL]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + tid + u * GTH;
                if (e < nb * M) {
                    const int r = e / nb, q = e - r * nb;
                    Pan[q * M + r] = v[u];
                }
            }
        }
        __syncthreads();
        // 1. partial pivoting on the panel.  Row r belongs to thread r mod GTH
        // for the whole panel, so a thread only ever reads rows it updated
        // itself, except the pivot row, which nobody writes once chosen.
        for (int q = 0; q < nb; ++q) {
            float best = -1.0f;
            int bidx = M;
            for (int r = tid; r < M; r += GTH)
                if (pstep[r] == M) {
                    const float2 v = Pan[q * M + r];
                    float a = fabsf(v.x) + fabsf(v.y);
                    if (!(a == a)) a = 3.0e38f;        // a NaN row is taken, so that ln det turns non-finite
                    if (a > best) { best = a; bidx = r; }
                }
            const int rs = gj_argmax(best, bidx, shv[par], shi[par]);
            par ^= 1;
            const float2 u = Pan[q * M + rs];
            if ((rs & (GTH - 1)) == tid) pstep[rs] = p + q;
            if (tid == 0) {
                piv[p + q] = rs;
                upiv[p + q] = u;
                ppiv[q] = rs;
                if (!(u.x * u.x + u.y * u.y > 0.0f)) atomicOr(status, 1);
            }
            const float n2 = u.x * u.x + u.y * u.y;
            const float2 ip = make_float2(u.x / n2, -u.y / n2);
            for (int r = tid; r < M; r += GTH)
                if (pstep[r] == M) {
                    const float2 l = cmul(Pan[q * M + r], ip);
                    Pan[q * M + r] = l;
                    for (int q2 = q + 1; q2 < nb; ++q2)
                        Pan[q2 * M + r] = csub_mul(Pan[q2 * M + r], l, Pan[q2 * M + rs]);
                }
        }
        __syncthreads();
        for (int e = tid; e < GNB * GNB; e += GTH) {
            const int q = e / GNB, q2 = e % GNB;
            LUpp[e] = (q < nb && q2 < nb) ? Pan[q2 * M + ppiv[q]] : make_float2(0.f, 0.f);
        }
        if (tid < GNB) {
            float2 v = make_float2(0.f, 0.f);
            if (tid < nb) {
                const float2 u = Pan[tid * M + ppiv[tid]];
                const float n2 = u.x * u.x + u.y * u.y;
                v = make_float2(u.x / n2, -u.y / n2);
            }
            ipv[tid] = v;
        }
        __syncthreads();

        for (int c0 = p + nb; c0 < 2 * M && !aborted; c0 += NT) {
            const int ncols = min(NT, 2 * M - c0);
            const int nmma = (ncols + 15) & ~15;
            // 2. R = P_pi^-1 S[pi, c], one column per thread
            if (tid < nmma) {
                const int c = c0 + tid;
                const bool cok = tid < ncols;
                float2 s[GNB];
#pragma unroll
                for (int q = 0; q < GNB; ++q) {
                    s[q] = make_float2(0.f, 0.f);
                    if (cok && q < nb) {
                        const float* a = re(ppiv[q], c);
                        s[q] = make_float2(a[0], a[PL]);
                    }
                }
#pragma unroll
                for (int q = 1; q < GNB; ++q) {          // unit lower triangle
                    float2 t = s[q];
#pragma unroll
                    for (int q2 = 0; q2 < q; ++q2) t = csub_mul(t, LUpp[q * GNB + q2], s[q2]);
                    s[q] = t;
                }
#pragma unroll
                for (int q = GNB - 1; q >= 0; --q) {     // upper triangle
                    float2 t = s[q];
#pragma unroll
                    for (int q2 = q + 1; q2 < GNB; ++q2) t = csub_mul(t, LUpp[q * GNB + q2], s[q2]);
                    s[q] = cmul(t, ipv[q]);
                }
#pragma unroll
                for (int q = 0; q < GNB; ++q)
                    if (cok && q < nb) {
                        float* a = re(ppiv[q], c);
                        a[0] = s[q].x;
                        a[PL] = s[q].y;
                    }
#pragma unroll
                for (int q = 0; q < GNB; ++q) {
                    put_split(Bhi, Blo, sw128_off(tid, q), s[q].x);
                    put_split(Bhi, Blo, sw128_off(tid, GNB + q), s[q].y);
                }
            }
            fence_async_smem();
            __syncthreads();
            // 3. rank-16 update of every other row, 64 complex rows per MMA tile
            for (int m0 = 0; m0 < M && !aborted; m0 += 64) {
                // this thread's epilogue entries: TMEM lane 32 (w mod 4) + lane =
                // (part, row r), chunks of 16 columns (w / 4) + 2 j.  Their old
                // values are loaded now, so that the loads are in flight during
                // the A build and the MMA.
                const int qd = wid & 3, Lr = 32 * qd + lane, part = Lr >> 6, re_r = m0 + (Lr & 63);
                const bool rok_e = re_r < M && !(pstep[re_r] >= p && pstep[re_r] < p + nb);
                const int nch = nmma >> 4;
                float sv[NCHW][16];
                float* rowp = Sw + (size_t)(rok_e ? re_r : 0) * RS + (size_t)part * PL;
#pragma unroll
                for (int j = 0; j < NCHW; ++j) {
                    const int cc = c0 + ((wid >> 2) + 2 * j) * 16;        // first column of the chunk
                    const bool vec = rok_e && (cc & 3) == 0 && cc + 16 <= c0 + ncols;
                    if (vec) {
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            const float4 v = *reinterpret_cast<const float4*>(rowp + cc + 4 * q4);
                            sv[j][4 * q4] = v.x;
                            sv[j][4 * q4 + 1] = v.y;
                            sv[j][4 * q4 + 2] = v.z;
                            sv[j][4 * q4 + 3] = v.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int c = cc + q;
                            sv[j][q] = (rok_e && c < c0 + ncols) ? rowp[c] : 0.f;
                        }
                    }
                }
                {
                    const int rl = tid & 63, r = m0 + rl;
                    const bool rok = r < M && !(pstep[r] >= p && pstep[r] < p + nb);
                    float2 av[GNB / 4];
#pragma unroll
                    for (int j = 0; j < GNB / 4; ++j) {
                        const int q = (tid >> 6) + 4 * j;
                        av[j] = make_float2(0.f, 0.f);
                        if (rok && q < nb) {
                            const float* a = re(r, p + q);
                            av[j] = make_float2(a[0], a[PL]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < GNB / 4; ++j) {
                        const int q = (tid >> 6) + 4 * j;
                        put_split(Ahi, Alo, sw128_off(rl, q), av[j].x);              // [Pr, -Pi]
                        put_split(Ahi, Alo, sw128_off(rl, GNB + q), -av[j].y);
                        put_split(Ahi, Alo, sw128_off(64 + rl, q), av[j].y);         // [Pi,  Pr]
                        put_split(Ahi, Alo, sw128_off(64 + rl, GNB + q), av[j].x);
                    }
                }
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint64_t ah = sdesc_sw128(Ahi), al = sdesc_sw128(Alo);
                    const uint64_t bh = sdesc_sw128(Bhi), bl = sdesc_sw128(Blo);
                    const uint32_t idesc = idesc_tf32(nmma);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t dk = (uint64_t)((k * 32) >> 4);   // 8 tf32 = 32 bytes along the row
                        mma_tf32(tmem, ah + dk, bh + dk, idesc, k > 0 ? 1u : 0u);
                        mma_tf32(tmem, ah + dk, bl + dk, idesc, 1u);
                        mma_tf32(tmem, al + dk, bh + dk, idesc, 1u);
                    }
                    mma_commit(&mbar);
                }
                const bool ok = mbar_wait(&mbar, phase & 1u, wait_limit);
                ++phase;
                if (!__syncthreads_and(ok)) {
                    aborted = true;
                    if (tid == 0) {
                        atomicOr(status, 2);
                        mbar_wait(&mbar, (phase - 1) & 1u);     // drain (default bound)
                    }
                    __syncthreads();
                    break;
                }
                tc_fence_after();
                const uint32_t tq = tmem + ((uint32_t)(32 * qd) << 16);
#pragma unroll
                for (int j = 0; j < NCHW; ++j) {
                    const int ch = (wid >> 2) + 2 * j;
                    if (ch < nch) {                               // uniform over the warp
                        uint32_t v[16];
                        tmem_ld16(tq + (uint32_t)(ch * 16), v);
                        if (rok_e) {
                            const int cc = c0 + ch * 16;
                            if ((cc & 3) == 0 && cc + 16 <= c0 + ncols) {
#pragma unroll
                                for (int q4 = 0; q4 < 4; ++q4)
                                    *reinterpret_cast<float4*>(rowp + cc + 4 * q4) =
                                        make_float4(sv[j][4 * q4] - __uint_as_float(v[4 * q4]),
                                                    sv[j][4 * q4 + 1] - __uint_as_float(v[4 * q4 + 1]),
                                                    sv[j][4 * q4 + 2] - __uint_as_float(v[4 * q4 + 2]),
                                                    sv[j][4 * q4 + 3] - __uint_as_float(v[4 * q4 + 3]));
                            } else {
#pragma unroll
                                for (int q = 0; q < 16; ++q)
                                    if (cc + q < c0 + ncols) rowp[cc + q] = sv[j][q] - __uint_as_float(v[q]);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncthreads();
            }
        }
    }

    if (!aborted) {
        double2 ldm = make_double2(0.0, 0.0);
        for (int j = tid; j < M; j += GTH) {
            const float2 u = upiv[j];
            const double ux = u.x, uy = u.y;
            ldm = ldm + make_double2(0.5 * log(ux * ux + uy * uy), atan2(uy, ux));
        }
        ldm = block_sum(ldm, shc);
        lsum = block_sum(lsum, shd);
        if (tid == 0) {
            // parity of the pivot order: M minus its number of cycles
            int cycles = 0;
            for (int s0 = 0; s0 < M; ++s0)
                if (pstep[s0] >= 0) {
                    ++cycles;
                    int x = s0;
                    while (x >= 0 && x < M && pstep[x] >= 0) {
                        const int nx = pstep[x];
                        pstep[x] = -1;
                        x = nx;
                    }
                }
            nswap_sh = (M - cycles) & 1;
        }
        // G[i][c] = delta_ic - S[pi_c][M + i] D_Ls[c]: rows pi_c of S are read
        // along i and G is written along c, through 32 x 33 shared tiles
        double2 trg = make_double2(0.0, 0.0);
        float2* tile = Pan;
        for (int cb = 0; cb < M; cb += 32)
            for (int ib = 0; ib < M; ib += 32) {
                float2 gv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = cb + wid + 8 * u, i = ib + lane;
                    gv[u] = make_float2(0.f, 0.f);
                    if (c < M && i < M) {
                        const float* a = re(piv[c], M + i);
                        gv[u] = make_float2(a[0], a[PL]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) tile[(wid + 8 * u) * 33 + lane] = gv[u];
                __syncthreads();
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = ib + wid + 8 * u, c = cb + lane;
                    if (c < M && i < M) {
                        const float2 x = tile[lane * 33 + wid + 8 * u];
                        float2 g = make_float2(-x.x * dls[c], -x.y * dls[c]);
                        if (c == i) {
                            g.x += 1.0f;
                            trg = trg + make_double2(g.x, g.y);
                        }
                        Gw[(size_t)i * M + c] = g;
                    }
                }
                __syncthreads();
            }
        trg = block_sum(trg, shc);
        if (tid == 0)
            green_weight_tail(ws + (long)WSTRIDE * w, ldm, lsum, nswap_sh, trg, M, kdt, constraint, status);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0) tmem_dealloc(tmem, (uint32_t)NT);
}

}  // namespace

size_t green_tc_smem(int M, int NT) { return GjLayout(M, NT).total; }

size_t green_tc_floats(int M) { return (size_t)M * 2 * gj_part_len(M); }

// N tile: 128 columns, or 64 when the layout would not fit; 0 when neither
// does.  At M = 257 the 128-column layout (111 KB) lets two walkers share an
// SM.
int green_tc_tile(int M) {
    for (int nt = NTMAX; nt >= 64; nt >>= 1)
        if (green_tc_smem(M, nt) <= 227 * 1024 - 4096) return nt;
    return 0;
}

cudaError_t launch_green_tc(ftq_ctx* c, int k, float2* G, double* ws) {
    const int M = c->M;
    const int NT = green_tc_tile(M);
    if (NT == 0) return cudaErrorInvalidValue;
    const size_t sm = green_tc_smem(M, NT);
    static size_t sm_set = 0;
    if (sm > sm_set) {
        cudaError_t e = cudaFuncSetAttribute(k_green_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        sm_set = sm;
    }
    Planes P;
    P.Kp = c->Kp;
    P.part = (size_t)c->LD * 2 * c->Kp;
    const long long wl = c->wait_limit >= 0 ? (long long)c->wait_limit : TC_WAIT_LIMIT;
    LaunchScope ls(c, FTQ_K_GREEN);
    k_green_tc<<<c->W, GTH, sm, c->stream>>>(c->Ypl, c->Tinv, c->DR, c->w32, G ? G : c->G32, c->tab.eps,
                                            ws ? ws : c->wstate,
                                            c->status, M, left_scale(c, k), c->sys.mu_T, c->opts.constraint, P,
                                            2 * P.part, (double)k * c->sys.dtau, NT, wl);
    return cudaGetLastError();
}

}  // namespace ftq

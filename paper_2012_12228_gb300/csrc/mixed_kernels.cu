// Mixed-precision slice path: the B chain held in FP32 planes split into
// tf32 hi + lo parts (the operand format of 3xTF32 tensor-core products),
// G(tau) and ln det per slice from an FP32 LU with FP64 log accumulation,
// and bridges to the complex128 QRCP (every s slices) and to the complex128
// G(beta) used by the estimators.
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"
#include "mixed_common.cuh"

namespace ftq {
namespace {

constexpr double kPi = 3.14159265358979323846;

template <typename T>
__device__ T block_sum(T v, T* sh) {
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

__device__ int block_argmax(float val, int idx, float* shv, int* shi) {
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_down_sync(0xffffffffu, val, o);
        int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { shv[wid] = val; shi[wid] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bv = shv[0];
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

// ---------------------------------------------------------------- layout bridges
__global__ void k_planes_identity(float* Ypl, int Kp, int M, size_t wstride, int W) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)W * M) return;
    int w = (int)(e / M), i = (int)(e % M);
    Ypl[wstride * w + (size_t)i * (2 * Kp) + i] = 1.0f;
}

__global__ void k_planes_to_c128(const float* __restrict__ Ypl, double2* __restrict__ Y, Planes P, int M,
                                 size_t wstride, long total) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    long w = e / ((long)M * M);
    int ij = (int)(e % ((long)M * M));
    int i = ij / M, c = ij % M;
    const float* p = Ypl + wstride * w;
    size_t o = (size_t)c * (2 * P.Kp) + i;
    Y[e] = make_double2((double)p[o] + (double)p[P.part + o], (double)p[o + P.Kp] + (double)p[P.part + o + P.Kp]);
}

// The complex128 chain (row-major) into the FP32 planes (tf32 hi + lo) and
// the single FP32 plane beside them: the low-rank stabilisation's new Q.
__global__ void k_c128_to_planes(const double2* __restrict__ Y, float* __restrict__ Ypl, float* __restrict__ Yf,
                                 Planes P, int M, size_t wstride, long total) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    long w = e / ((long)M * M);
    int ij = (int)(e % ((long)M * M));
    int i = ij / M, c = ij % M;
    const double2 y = Y[e];
    const float2 v = make_float2((float)y.x, (float)y.y);
    P.store(Ypl + wstride * w, i, c, v);
    float* f = Yf + P.part * w + (size_t)c * (2 * P.Kp) + i;
    f[0] = v.x;
    f[P.Kp] = v.y;
}

__global__ void k_c64_to_c128(const float2* __restrict__ a, double2* __restrict__ b, long total) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    float2 v = a[e];
    b[e] = make_double2(v.x, v.y);
}

__global__ void k_g32_init(float2* G, const double* g0, int M, long total) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    int ij = (int)(e % ((long)M * M));
    int i = ij / M, j = ij % M;
    G[e] = make_float2(i == j ? (float)g0[i] : 0.0f, 0.0f);
}

// ---------------------------------------------------------------- FP32 chain (CUDA cores)
// out = os (us Y + alpha V (zs Z)) on the split planes; V gathered from phi.
constexpr int ST = 64;   // output tile (complex)
constexpr int SK = 16;   // k tile

__global__ void __launch_bounds__(256) k_chain32(const float* __restrict__ Zin, const float* __restrict__ Yu,
                                                float* __restrict__ out, const double2* __restrict__ phi,
                                                const uint16_t* __restrict__ vidx, const double* __restrict__ zs,
                                                const double* __restrict__ us, const double* __restrict__ os,
                                                float alpha, int M, int nslot, int tiles, Planes P, size_t wstride) {
    __shared__ float2 As[SK][ST + 1];
    __shared__ float2 Bs[SK][ST + 1];
    const int w = blockIdx.y;
    const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles;
    const int r0 = ti * ST, c0 = tj * ST;
    const float* Z = Zin + wstride * w;
    const double2* ph = phi + (long)w * nslot;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < M; k0 += SK) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            int e = threadIdx.x + 256 * l;          // 0..1023
            int r = e >> 4, kk = e & 15;            // A: 64 rows x 16 k
            int i = r0 + r, k = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (i < M && k < M) {
                double2 d = ph[vidx[(long)i * M + k]];
                double s = zs ? zs[k] : 1.0;
                v = make_float2((float)(d.x * s), (float)(d.y * s));
            }
            As[kk][r] = v;
            int kb = e >> 6, cb = e & 63;           // B: 16 k x 64 cols
            int kr = k0 + kb, cc = c0 + cb;
            float2 z = make_float2(0.f, 0.f);
            if (kr < M && cc < M) z = P.load(Z, kr, cc);
            Bs[kb][cb] = z;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = cfma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
    float* O = out + wstride * w;
    const float* U = Yu + wstride * w;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int i = r0 + ty + 16 * a, c = c0 + tx + 16 * b;
            if (i < M && c < M) {
                float2 u = P.load(U, i, c);
                const ScaleF s(us[i]);
                float2 v = make_float2(fmaf(alpha, acc[a][b].x, s(u.x)), fmaf(alpha, acc[a][b].y, s(u.y)));
                if (os) {
                    const ScaleF o(os[i]);
                    v.x = o(v.x);
                    v.y = o(v.y);
                }
                P.store(O, i, c, v);
            }
        }
}

// ---------------------------------------------------------------- FP32 G(tau) + ln det
// Same algebra as the complex128 kernel: Mt = D_Lb T^-1 D_Rb + D_Ls Y D_Rs in
// FP32, LU with partial pivoting, G = I - Y D_Rs Mt^-1 D_Ls, ln det from the
// pivots accumulated in FP64, weight update in FP64.
__global__ void k_green32(const float* __restrict__ Ypl, const double2* __restrict__ Tinv,
                          const double2* __restrict__ DR, float2* __restrict__ work, float2* __restrict__ work2,
                          float2* __restrict__ G, const double* __restrict__ eps, double* __restrict__ ws,
                          int* __restrict__ status, int M, double lscale, double mu_T, int constraint,
                          Planes P, size_t wstride, double kdt) {
    extern __shared__ unsigned char smem_raw[];
    float2* drs = reinterpret_cast<float2*>(smem_raw);      // [M]
    float2* invU = drs + M;                                 // [M]
    float* dls = reinterpret_cast<float*>(invU + M);        // [M]
    float* dlb = dls + M;                                   // [M]
    float* drb = dlb + M;                                   // [M]
    int* perm = reinterpret_cast<int*>(drb + M);            // [M]
    __shared__ float shv[32];
    __shared__ int shi[32];
    __shared__ double shd[32];
    __shared__ double2 shc[32];
    __shared__ int nswap;
    const int w = blockIdx.x;
    const long off = (long)w * M * M;
    const int nt = blockDim.x;
    float2* A = work + off;
    float2* XT = work2 + off;
    const float* Yw = Ypl + wstride * w;
    const double2* Tw = Tinv + off;
    float2* Gw = G + off;

    double lsum = 0.0;
    for (int i = threadIdx.x; i < M; i += nt) {
        double dl = exp(-lscale * (eps[i] - mu_T));
        double b, s2;
        if (dl > 1.0) { b = 1.0 / dl; s2 = 1.0; } else { b = 1.0; s2 = dl; }
        dlb[i] = (float)b; dls[i] = (float)s2;
        double2 d = DR[(long)w * M + i];
        double a = sqrt(abs2(d));
        double rb;
        double2 rs;
        if (a > 1.0) { rb = 1.0 / a; rs = d * (1.0 / a); } else { rb = 1.0; rs = d; }
        drb[i] = (float)rb;
        drs[i] = make_float2((float)rs.x, (float)rs.y);
        lsum += log(b) + log(rb);
        perm[i] = i;
    }
    if (threadIdx.x == 0) nswap = 0;
    __syncthreads();
    for (long e = threadIdx.x; e < (long)M * M; e += nt) {
        int i = (int)(e / M), j = (int)(e % M);
        double2 t = Tw[e] * ((double)dlb[i] * (double)drb[j]);
        float2 y = cmul(P.load(Yw, i, j), drs[j]) * dls[i];
        A[e] = make_float2((float)t.x + y.x, (float)t.y + y.y);
    }
    __syncthreads();
    for (int j = 0; j < M; ++j) {
        float best = -1.0f;
        int bidx = M;
        for (int i = j + threadIdx.x; i < M; i += nt) {
            float2 v = A[(long)i * M + j];
            float a1 = fabsf(v.x) + fabsf(v.y);
            if (a1 > best) { best = a1; bidx = i; }
        }
        int p = block_argmax(best, bidx, shv, shi);
        if (p >= M) {
            p = j;
            if (threadIdx.x == 0) atomicOr(status, 1);
        }
        if (p != j) {
            for (int c = threadIdx.x; c < M; c += nt) {
                float2 t = A[(long)j * M + c];
                A[(long)j * M + c] = A[(long)p * M + c];
                A[(long)p * M + c] = t;
            }
            if (threadIdx.x == 0) {
                int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
                nswap ^= 1;
            }
        }
        __syncthreads();
        const float2 piv = A[(long)j * M + j];
        const float n2 = piv.x * piv.x + piv.y * piv.y;
        if (!(n2 > 0.0f) && threadIdx.x == 0) atomicOr(status, 1);
        const float2 ip = make_float2(piv.x / n2, -piv.y / n2);
        for (int i = j + 1 + threadIdx.x; i < M; i += nt) A[(long)i * M + j] = cmul(A[(long)i * M + j], ip);
        if (threadIdx.x == 0) invU[j] = ip;
        __syncthreads();
        for (int c = j + 1 + threadIdx.x; c < M; c += nt) {
            const float2 u = A[(long)j * M + c];
            for (int i = j + 1; i < M; ++i) A[(long)i * M + c] = A[(long)i * M + c] - cmul(A[(long)i * M + j], u);
        }
        __syncthreads();
    }
    double2 ldm = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < M; j += nt) {
        float2 u = A[(long)j * M + j];
        double ux = u.x, uy = u.y;
        ldm = ldm + make_double2(0.5 * log(ux * ux + uy * uy), atan2(uy, ux));
    }
    ldm = block_sum(ldm, shc);
    lsum = block_sum(lsum, shd);
    for (int i = threadIdx.x; i < M; i += nt) {
        for (int j = 0; j < M; ++j) {
            float2 s = cmul(P.load(Yw, i, j), drs[j]);
            for (int m = 0; m < j; ++m) s = s - cmul(XT[(long)m * M + i], A[(long)m * M + j]);
            XT[(long)j * M + i] = cmul(s, invU[j]);
        }
        for (int j = M - 2; j >= 0; --j) {
            float2 s = XT[(long)j * M + i];
            for (int m = j + 1; m < M; ++m) s = s - cmul(XT[(long)m * M + i], A[(long)m * M + j]);
            XT[(long)j * M + i] = s;
        }
        for (int m = 0; m < M; ++m) {
            int c = perm[m];
            float2 g = XT[(long)m * M + i] * (-dls[c]);
            if (c == i) g.x += 1.0f;
            Gw[(long)i * M + c] = g;
        }
    }
    __syncthreads();
    double2 trg = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const float2 g = Gw[(long)i * M + i];
        trg = trg + make_double2(g.x, g.y);
    }
    trg = block_sum(trg, shc);
    if (threadIdx.x == 0) {
        double* s = ws + (long)WSTRIDE * w;
        double2 ld = ldm;
        ld.x -= lsum;
        ld.y += kPi * (double)(nswap ^ ((int)s[7]));
        if (!isfinite(ld.x) || !isfinite(ld.y)) atomicOr(status, 1);
        // d ln det(I + A_k)/dmu = k dtau (M - tr G(tau_k)): every B carries exp(dtau mu)
        const double2 tk = make_double2(kdt * ((double)M - trg.x), -kdt * trg.y);
        const double2 dlnS = make_double2(2.0 * (tk.x - s[9]), 2.0 * (tk.y - s[10]));
        double2 lnS = make_double2(2.0 * (ld.x - s[3]), 2.0 * (ld.y - s[4]));
        double gr = s[5], gi = s[6];
        if (constraint == FTQ_FREE) {
            s[0] += lnS.x + gr;
            s[1] = remainder(s[1] + lnS.y + gi, 2.0 * kPi);
            s[8] += dlnS.x;
            s[11] += dlnS.y;
        } else if (s[2] > 0.5) {
            const double cth = cos(lnS.y);
            if (!isfinite(lnS.x + gr) || !(cth == cth)) {
                // a non-finite ratio or Gaussian factor drops the walker (weight 0)
                s[2] = 0.0;
                atomicOr(status, 1);
            } else if (cth <= 0.0) {
                s[2] = 0.0;
            } else {
                s[0] += lnS.x + gr + log(cth);
                s[8] += dlnS.x - tan(lnS.y) * dlnS.y;   // d log cos(theta) = -tan(theta) d theta
            }
        }
        s[3] = ld.x;
        s[4] = remainder(ld.y, 2.0 * kPi);
        s[9] = tk.x;
        s[10] = tk.y;
    }
}

int fact_threads(int M) {
    int t = ((M + 31) / 32) * 32;
    return t > 1024 ? 1024 : (t < 32 ? 32 : t);
}

Planes planes_of(const ftq_ctx* c) {
    Planes P;
    P.Kp = c->Kp;
    P.part = (size_t)c->LD * 2 * c->Kp;
    return P;
}

size_t walker_stride(const ftq_ctx* c) { return 2 * (size_t)c->LD * 2 * c->Kp; }

}  // namespace

cudaError_t mixed_init(ftq_ctx* c) {
    const int M = c->M, W = c->W;
    const size_t ws = walker_stride(c);
    cudaError_t e = cudaMemsetAsync(c->Ypl, 0, sizeof(float) * ws * W, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->Yf, 0, sizeof(float) * (ws / 2) * W, c->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(c->zpl[b], 0, sizeof(float) * ws * W, c->stream);
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls(c, FTQ_K_INIT);
        long n = (long)W * M;
        k_planes_identity<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->Ypl, c->Kp, M, ws, W);
        k_planes_identity<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->Yf, c->Kp, M, ws / 2, W);
    }
    {
        LaunchScope ls(c, FTQ_K_INIT);
        long n = (long)W * M * M;
        k_g32_init<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->G32, c->tab.g0, M, n);
    }
    c->g64_valid = true;
    return cudaGetLastError();
}

cudaError_t mixed_chain(ftq_ctx* c) {
    const int M = c->M, p = c->opts.exp_order;
    const bool tensor = c->opts.precision == FTQ_MIXED || c->opts.precision == FTQ_MIXED_F64UDT;
    const int tiles = (M + ST - 1) / ST;
    dim3 grid(tiles * tiles, c->W);
    const Planes P = planes_of(c);
    const size_t ws = walker_stride(c);
    const float* zin = c->Ypl;
    int cur = 0;
    for (int j = p; j >= 1; --j) {
        float* out = c->zpl[cur];
        const double* zs = j == p ? c->tab.h : nullptr;
        const double* os = j == 1 ? c->tab.h : nullptr;
        if (tensor) {
            cudaError_t e = tc_chain_step(c, zin, out, zs, os, 1.0f / j);
            if (e != cudaSuccess) return e;
        } else {
            LaunchScope ls(c, FTQ_K_CHAIN);
            k_chain32<<<grid, 256, 0, c->stream>>>(zin, c->Ypl, out, c->phi, c->tab.vidx, zs, c->tab.h, os,
                                                   1.0f / j, M, c->nslot, tiles, P, ws);
        }
        zin = out;
        cur ^= 1;
    }
    float* res = c->zpl[cur ^ 1];
    c->zpl[cur ^ 1] = c->Ypl;
    c->Ypl = res;
    return cudaGetLastError();
}

// The mixed chain as complex128 in c->Y (the low-rank path's factorisations
// run in complex128 on it).
cudaError_t planes_to_y64(ftq_ctx* c) {
    const long n = (long)c->W * c->M * c->M;
    LaunchScope ls(c, FTQ_K_BRIDGE);
    k_planes_to_c128<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->Ypl, c->Y, planes_of(c), c->M,
                                                                     walker_stride(c), n);
    return cudaGetLastError();
}

cudaError_t mixed_qrcp(ftq_ctx* c) {
    if (c->opts.low_rank_threshold <= 0.0) return launch_qr_prepiv(c);
    // low rank (Eq. thresh): the pivoted QR of the M x m panel and the
    // truncation in complex128 on the chain's copy, the new Q back into the
    // FP32 planes, and the tensor-core work list cut to the new ranks
    cudaError_t e = planes_to_y64(c);
    if (e == cudaSuccess) e = launch_qrcp_lr(c);            // c->Y <- Q, ranks -> ws[12]
    if (e != cudaSuccess) return e;
    {
        const long n = (long)c->W * c->M * c->M;
        LaunchScope ls(c, FTQ_K_BRIDGE);
        k_c128_to_planes<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->Y, c->Ypl, c->Yf, planes_of(c),
                                                                          c->M, walker_stride(c), n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && c->opts.precision == FTQ_MIXED) e = tc_items_by_rank(c);
    return e;
}

cudaError_t mixed_green(ftq_ctx* c, int k) {
    const int M = c->M;
    if (c->opts.low_rank_threshold > 0.0) {
        // low rank: G(tau_k) and ln det by the Woodbury form in complex128 on
        // the chain's copy (O(M m m_L) per walker), every slice
        cudaError_t e = planes_to_y64(c);
        if (e == cudaSuccess) e = launch_green64(c, c->Y, k, true);
        if (e == cudaSuccess && k == c->sys.n_slices && c->opts.overlap == FTQ_OVERLAP_MODIFIED)
            e = launch_green64(c, c->Y, k, true, true);
        c->g64_valid = true;
        return e;
    }
    if (k == c->sys.n_slices) {
        // tau = beta: the final G and ln det in complex128
        const long n = (long)c->W * M * M;
        {
            LaunchScope ls(c, FTQ_K_BRIDGE);
            k_planes_to_c128<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                c->Ypl, c->zbuf[1], planes_of(c), M, walker_stride(c), n);
        }
        cudaError_t e = launch_green64(c, c->zbuf[1], k, true);
        if (e == cudaSuccess && c->opts.overlap == FTQ_OVERLAP_MODIFIED)
            e = launch_green64(c, c->zbuf[1], k, true, true);
        c->g64_valid = true;
        return e;
    }
    if (green_uses_tc(c)) {
        // rank-16 Gauss-Jordan updates on the tensor cores
        cudaError_t e = launch_green_tc(c, k);
        c->g64_valid = false;
        return e;
    }
    if (green32b_smem(M) <= 220 * 1024) {
        cudaError_t e = launch_green32b(c, k);
        c->g64_valid = false;
        return e;
    }
    size_t sm = (2 * sizeof(float2) + 3 * sizeof(float) + sizeof(int)) * M;
    int nt = fact_threads(M);
    double lscale = left_scale(c, k);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_green32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    LaunchScope ls(c, FTQ_K_GREEN);
    k_green32<<<c->W, nt, sm, c->stream>>>(c->Ypl, c->Tinv, c->DR, c->w32, c->w2_32, c->G32, c->tab.eps, c->wstate,
                                          c->status, M, lscale, c->sys.mu_T, c->opts.constraint, planes_of(c),
                                          walker_stride(c), (double)k * c->sys.dtau);
    c->g64_valid = false;
    return cudaGetLastError();
}

// Which Green kernel the mixed path runs for slices k < n.  The tensor-core
// Gauss-Jordan kernel streams S = [Mt^T | B^T] once per 16-column panel, the
// CUDA-core blocked LU computes in shared-memory panels with four walkers per
// SM; measured per 5-slice block on a GB300: M = 257, 1024 walkers: 96.7 ms
// (tensor cores) vs 63.6 ms (LU); M = 515, 152 walkers: 86.5 vs 149.1 ms.
// Without a measurement the crossover is taken between the two basis sizes;
// ftq_autotune times both on the context's own workload.
constexpr int GREEN_TC_MIN_M = 384;

bool green_uses_tc(const ftq_ctx* c) {
    if (c->opts.precision == FTQ_MIXED_SIMT || green_tc_tile(c->M) == 0) return false;
    if (c->green_kind == 1) return true;
    if (c->green_kind == 2) return false;
    return c->M >= GREEN_TC_MIN_M;
}

// Time one launch of each Green kernel (after one warm-up launch) on the
// context's current chain, writing G and the weights into scratch buffers
// (zbuf[0] and est), so that neither G(tau) nor the walker state changes.
cudaError_t green_autotune(ftq_ctx* c, float* ms_tc, float* ms_lu) {
    *ms_tc = *ms_lu = 0.f;
    if (c->opts.precision == FTQ_MIXED_SIMT || c->opts.low_rank_threshold > 0.0 || green_tc_tile(c->M) == 0)
        return cudaSuccess;
    float2* gs = reinterpret_cast<float2*>(c->zbuf[0]);
    double* ws = c->est;
    const size_t wbytes = sizeof(double) * WSTRIDE * (size_t)c->W;
    int saved_status = 0;
    cudaError_t e = cudaMemcpyAsync(&saved_status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int k = c->k < c->sys.n_slices ? c->k + 1 : 1;
    for (int kind = 1; kind <= 2 && e == cudaSuccess; ++kind) {
        auto run = [&]() { return kind == 1 ? launch_green_tc(c, k, gs, ws) : launch_green32b(c, k, gs, ws); };
        e = cudaMemcpyAsync(ws, c->wstate, wbytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = run();                          // warm-up
        if (e == cudaSuccess) e = cudaMemcpyAsync(ws, c->wstate, wbytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        (kind == 1 ? *ms_tc : *ms_lu) = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the trial inputs are whatever the chain holds; a flag they raise is not the caller's
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->status, &saved_status, sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) c->green_kind = *ms_tc < *ms_lu ? 1 : 2;
    return e;
}

cudaError_t mixed_sync_g64(ftq_ctx* c) {
    const long n = (long)c->W * c->M * c->M;
    k_c64_to_c128<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->G32, c->G, n);
    c->launches[FTQ_K_BRIDGE] += 1;
    c->g64_valid = true;
    return cudaGetLastError();
}

}  // namespace ftq

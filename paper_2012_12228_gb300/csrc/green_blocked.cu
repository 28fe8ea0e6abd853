// Blocked FP32 Green's function of the mixed path: the same algebra as the
// complex128 kernel (Mt = D_Lb T^-1 D_Rb + D_Ls Y D_Rs, LU with partial
// pivoting, G(tau) = I - Y D_Rs Mt^-1 D_Ls, ln det accumulated in FP64),
// organised so that almost all flops are register-tiled updates from
// shared memory instead of streams through L2:
//
//   LU: 32-column panels factorised in shared memory; the row swaps are
//       applied to the rest of the matrix column by column; U12 = L11^-1 A12
//       one column per thread; A22 -= L21 U12 in 4 x 4 complex micro-tiles.
//   X U = Y D_Rs and W L = X: 32-column blocks, one row per thread, the
//       block of U (or L) staged in shared memory and broadcast.
//
// One thread block per walker (ceil(M/32) warps, 256..384 threads, so that
// the solves take one row per thread); matrices live in L2 / HBM.
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"
#include "mixed_common.cuh"

namespace ftq {
namespace {

constexpr int NB = 32;
constexpr int GT_MAX = 384;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ float2 csub_mul(float2 acc, float2 a, float2 b) {
    // acc - a * b
    return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}

template <typename T>
__device__ T bsum(T v, T* sh) {
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_down(v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        T acc = sh[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) acc = acc + sh[i];
        sh[0] = acc;
    }
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

__device__ int bargmax(float val, int idx, float* shv, int* shi) {
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
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            if (shv[i] > bv || (shv[i] == bv && shi[i] < bi)) { bv = shv[i]; bi = shi[i]; }
        shi[0] = bi;
    }
    __syncthreads();
    int r = shi[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(GT_MAX, 1) k_green32b(const float* __restrict__ Ypl, const double2* __restrict__ Tinv,
                                                   const double2* __restrict__ DR, float2* __restrict__ work,
                                                   float2* __restrict__ work2, float2* __restrict__ G,
                                                   const double* __restrict__ eps, double* __restrict__ ws,
                                                   int* __restrict__ status, int M, double lscale, double mu_T,
                                                   int constraint, Planes P, size_t wstride, double kdt) {
    extern __shared__ unsigned char smem_raw[];
    float2* Ps = reinterpret_cast<float2*>(smem_raw);        // [M][NB]  panel / staged triangle block
    float2* Us = Ps + (size_t)M * NB;                          // [NB][M]  U12 rows of the current panel
    float2* drs = Us + (size_t)NB * M;                         // [M]
    float2* invU = drs + M;                                    // [M]
    float* dls = reinterpret_cast<float*>(invU + M);           // [M]
    float* dlb = dls + M;                                      // [M]
    float* drb = dlb + M;                                      // [M]
    int* perm = reinterpret_cast<int*>(drb + M);               // [M]
    int* piv = perm + M;                                       // [M]
    __shared__ float shv[32];
    __shared__ int shi[32];
    __shared__ double shd[32];
    __shared__ double2 shc[32];
    __shared__ int nswap;
    const int tid = threadIdx.x;
    const int GT = blockDim.x;
    const int w = blockIdx.x;
    const long off = (long)w * M * M;
    float2* A = work + off;
    float2* X = work2 + off;
    const float* Yw = Ypl + wstride * w;
    const double2* Tw = Tinv + off;
    float2* Gw = G + off;

    double lsum = 0.0;
    for (int i = tid; i < M; i += GT) {
        double dl = exp(-lscale * (eps[i] - mu_T));
        double b, s2;
        if (dl > 1.0) { b = 1.0 / dl; s2 = 1.0; } else { b = 1.0; s2 = dl; }
        dlb[i] = (float)b;
        dls[i] = (float)s2;
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
    if (tid == 0) nswap = 0;
    __syncthreads();
    for (long e = tid; e < (long)M * M; e += GT) {
        int i = (int)(e / M), j = (int)(e % M);
        double2 t = Tw[e] * ((double)dlb[i] * (double)drb[j]);
        float2 y = cmul(P.load(Yw, i, j), drs[j]) * dls[i];
        A[e] = make_float2((float)t.x + y.x, (float)t.y + y.y);
    }
    __syncthreads();

    // ---------------------------------------------------------------- blocked LU
    for (int jb = 0; jb < M; jb += NB) {
        const int nb = min(NB, M - jb);
        const int rows = M - jb;
        for (int e = tid; e < rows * nb; e += GT) {
            const int r = e / nb, c = e % nb;
            Ps[r * NB + c] = A[(long)(jb + r) * M + jb + c];
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            float best = -1.0f;
            int bidx = M;
            for (int r = j + tid; r < rows; r += GT) {
                const float2 v = Ps[r * NB + j];
                const float a1 = fabsf(v.x) + fabsf(v.y);
                if (a1 > best) { best = a1; bidx = r; }
            }
            int p = bargmax(best, bidx, shv, shi);
            if (p >= rows) {
                p = j;
                if (tid == 0) atomicOr(status, 1);
            }
            if (p != j)
                for (int c = tid; c < nb; c += GT) {
                    const float2 t = Ps[j * NB + c];
                    Ps[j * NB + c] = Ps[p * NB + c];
                    Ps[p * NB + c] = t;
                }
            if (tid == 0) piv[jb + j] = jb + p;
            __syncthreads();
            const float2 pv = Ps[j * NB + j];
            const float n2 = pv.x * pv.x + pv.y * pv.y;
            if (!(n2 > 0.0f) && tid == 0) atomicOr(status, 1);
            const float2 ip = make_float2(pv.x / n2, -pv.y / n2);
            if (tid == 0) invU[jb + j] = ip;
            for (int r = j + 1 + tid; r < rows; r += GT) Ps[r * NB + j] = cmul(Ps[r * NB + j], ip);
            __syncthreads();
            const int nr = rows - j - 1, nc = nb - j - 1;
            for (int e = tid; e < nr * nc; e += GT) {
                const int r = j + 1 + e / nc, c = j + 1 + e % nc;
                Ps[r * NB + c] = csub_mul(Ps[r * NB + c], Ps[r * NB + j], Ps[j * NB + c]);
            }
            __syncthreads();
        }
        for (int e = tid; e < rows * nb; e += GT) {
            const int r = e / nb, c = e % nb;
            A[(long)(jb + r) * M + jb + c] = Ps[r * NB + c];
        }
        // the panel's row interchanges on every other column, in order
        for (int c = tid; c < M; c += GT) {
            if (c >= jb && c < jb + nb) continue;
            for (int j = 0; j < nb; ++j) {
                const int r1 = jb + j, r2 = piv[jb + j];
                if (r1 != r2) {
                    const float2 t = A[(long)r1 * M + c];
                    A[(long)r1 * M + c] = A[(long)r2 * M + c];
                    A[(long)r2 * M + c] = t;
                }
            }
        }
        if (tid == 0)
            for (int j = 0; j < nb; ++j) {
                const int r2 = piv[jb + j];
                if (r2 != jb + j) {
                    const int t = perm[jb + j];
                    perm[jb + j] = perm[r2];
                    perm[r2] = t;
                    nswap ^= 1;
                }
            }
        __syncthreads();
        // U12 = L11^-1 A12, one column per thread
        const int c0 = jb + nb;
        const int ncr = M - c0;
        for (int c = tid; c < ncr; c += GT) {
            float2 x[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) x[q] = A[(long)(jb + q) * M + c0 + c];
#pragma unroll
            for (int q = 1; q < NB; ++q)
                if (q < nb) {
                    float2 s = x[q];
#pragma unroll
                    for (int q2 = 0; q2 < NB; ++q2)
                        if (q2 < q) s = csub_mul(s, Ps[q * NB + q2], x[q2]);
                    x[q] = s;
                }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) {
                    A[(long)(jb + q) * M + c0 + c] = x[q];
                    Us[q * M + c] = x[q];
                }
        }
        __syncthreads();
        // A22 -= L21 U12 in 4 x 4 micro-tiles (rows and columns strided so
        // that a warp reads consecutive columns)
        const int nrr = M - c0;
        if (nrr > 0) {
            const int tr = (nrr + 3) / 4, tc = (ncr + 3) / 4;
            for (int t = tid; t < tr * tc; t += GT) {
                const int rg = t / tc, cg = t % tc;
                float2 acc[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int r = rg + x * tr, c = cg + y * tc;
                        acc[x][y] = (r < nrr && c < ncr) ? A[(long)(c0 + r) * M + c0 + c] : make_float2(0.f, 0.f);
                    }
                for (int k = 0; k < nb; ++k) {
                    float2 a[4], b[4];
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const int r = rg + x * tr;
                        a[x] = r < nrr ? Ps[(nb + r) * NB + k] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int c = cg + y * tc;
                        b[y] = c < ncr ? Us[k * M + c] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] = csub_mul(acc[x][y], a[x], b[y]);
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int r = rg + x * tr, c = cg + y * tc;
                        if (r < nrr && c < ncr) A[(long)(c0 + r) * M + c0 + c] = acc[x][y];
                    }
            }
        }
        __syncthreads();
    }
    double2 ldm = make_double2(0.0, 0.0);
    for (int j = tid; j < M; j += GT) {
        const float2 u = A[(long)j * M + j];
        const double ux = u.x, uy = u.y;
        ldm = ldm + make_double2(0.5 * log(ux * ux + uy * uy), atan2(uy, ux));
    }
    ldm = bsum(ldm, shc);
    lsum = bsum(lsum, shd);

    // ---------------------------------------------------------------- X U = Y D_Rs
    for (int jb = 0; jb < M; jb += NB) {
        const int nb = min(NB, M - jb);
        for (int e = tid; e < (jb + nb) * nb; e += GT) {
            const int m = e / nb, q = e % nb;
            Ps[m * NB + q] = A[(long)m * M + jb + q];
        }
        __syncthreads();
        for (int i = tid; i < M; i += GT) {
            float2 s[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) s[q] = cmul(P.load(Yw, i, jb + q), drs[jb + q]);
            for (int m = 0; m < jb; ++m) {
                const float2 x = X[(long)i * M + m];
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (q < nb) s[q] = csub_mul(s[q], x, Ps[m * NB + q]);
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) {
                    float2 t = s[q];
#pragma unroll
                    for (int q2 = 0; q2 < NB; ++q2)
                        if (q2 < q) t = csub_mul(t, s[q2], Ps[(jb + q2) * NB + q]);
                    s[q] = cmul(t, invU[jb + q]);
                }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) X[(long)i * M + jb + q] = s[q];
        }
        __syncthreads();
    }
    // ---------------------------------------------------------------- W L = X (in place)
    const int nblk = (M + NB - 1) / NB;
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int jb = bi * NB;
        const int nb = min(NB, M - jb);
        for (int e = tid; e < (M - jb) * nb; e += GT) {
            const int m = jb + e / nb, q = e % nb;
            Ps[(m - jb) * NB + q] = A[(long)m * M + jb + q];
        }
        __syncthreads();
        for (int i = tid; i < M; i += GT) {
            float2 s[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) s[q] = X[(long)i * M + jb + q];
            for (int m = jb + nb; m < M; ++m) {
                const float2 x = X[(long)i * M + m];
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (q < nb) s[q] = csub_mul(s[q], x, Ps[(m - jb) * NB + q]);
            }
#pragma unroll
            for (int q = NB - 2; q >= 0; --q)
                if (q < nb - 1) {
                    float2 t = s[q];
#pragma unroll
                    for (int q2 = 1; q2 < NB; ++q2)
                        if (q2 > q && q2 < nb) t = csub_mul(t, s[q2], Ps[q2 * NB + q]);
                    s[q] = t;
                }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) X[(long)i * M + jb + q] = s[q];
        }
        __syncthreads();
    }
    // G[i][perm[m]] = delta - W[i][m] dls[perm[m]]
    for (int i = tid; i < M; i += GT)
        for (int m = 0; m < M; ++m) {
            const int c = perm[m];
            float2 g = X[(long)i * M + m] * (-dls[c]);
            if (c == i) g.x += 1.0f;
            Gw[(long)i * M + c] = g;
        }
    __syncthreads();
    double2 trg = make_double2(0.0, 0.0);
    for (int i = tid; i < M; i += GT) {
        const float2 g = Gw[(long)i * M + i];
        trg = trg + make_double2(g.x, g.y);
    }
    trg = bsum(trg, shc);
    if (tid == 0) {
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
            double cth = cos(lnS.y);
            if (cth <= 0.0) {
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

}  // namespace

size_t green32b_smem(int M) {
    return (size_t)M * NB * sizeof(float2) * 2 + (size_t)M * (2 * sizeof(float2) + 3 * sizeof(float) + 2 * sizeof(int));
}

cudaError_t launch_green32b(ftq_ctx* c, int k) {
    const int M = c->M;
    const size_t sm = green32b_smem(M);
    static size_t sm_set = 0;
    if (sm > sm_set) {
        cudaError_t e = cudaFuncSetAttribute(k_green32b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        sm_set = sm;
    }
    Planes P;
    P.Kp = c->Kp;
    P.part = (size_t)c->LD * 2 * c->Kp;
    const double lscale = (double)(c->sys.n_slices - k) * c->sys.dtau;
    int nt = (M + 31) / 32 * 32;
    nt = nt < 256 ? 256 : (nt > GT_MAX ? GT_MAX : nt);
    LaunchScope ls(c, FTQ_K_GREEN);
    k_green32b<<<c->W, nt, sm, c->stream>>>(c->Ypl, c->Tinv, c->DR, c->w32, c->w2_32, c->G32, c->tab.eps, c->wstate,
                                           c->status, M, lscale, c->sys.mu_T, c->opts.constraint, P, 2 * P.part,
                                           (double)k * c->sys.dtau);
    return cudaGetLastError();
}

}  // namespace ftq

// Blocked FP32 Green's function of the mixed path: the same algebra as the
// complex128 kernel (Mt = D_Lb T^-1 D_Rb + D_Ls Y D_Rs, LU with partial
// pivoting, G(tau) = I - Y D_Rs Mt^-1 D_Ls, ln det accumulated in FP64),
// organised so that almost all flops are register-tiled updates from
// shared memory instead of streams through L2:
//
//   LU: NB-column panels factorised in shared memory; the row swaps are
//       applied to the rest of the matrix column by column; U12 = L11^-1 A12
//       one column per thread; A22 -= L21 U12 in 3 x 3 complex micro-tiles.
//   X U = Y D_Rs and W L = X: NB-column blocks, one row per thread, the
//       block of U (or L) staged in shared memory and broadcast; X is stored
//       column-major so that a warp's loads of one column are contiguous.
//   G is written through 32 x 33 shared tiles with the inverse pivot order.
//
// One thread block per walker (ceil(M/32) warps, 256..288 threads, so that
// the solves take one row per thread); matrices live in L2 / HBM.  The kernel
// is latency-bound, so the panel width (NB = 8) and the register cap are
// chosen for occupancy: four walkers per SM (a measured sweep over NB = 4, 8,
// 16, 32 and one to five blocks per SM at M = 257).  At that occupancy the
// cap is 56 registers, and local-memory spills cost more than the shared
// reads a larger micro-tile saves: values only thread 0 needs at the end are
// parked in shared memory, and the hot loops carry no guards they can do
// without.
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"
#include "green_tail.cuh"
#include "mixed_common.cuh"

namespace ftq {
namespace {

constexpr int NB = 8;
constexpr int SU = 8;          // rows of X loaded per step of the solves (loads in flight per thread)
constexpr int TX = 3, TY = 3;  // complex micro-tile of the LU trailing update (fastest measured, 1x8 to 4x4)
constexpr int PSTR = NB + 1;   // padded row stride of the LU panel (column reads conflict-free)
constexpr int TILE = 32 * 33;  // one padded 32 x 32 transpose tile

// Length of the U12 region, which also holds the transpose tile.
__host__ __device__ __forceinline__ int us_len(int M) { return NB * M > TILE ? NB * M : TILE; }
constexpr int GT_MAX = 288;

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

// Block-wide argmax (ties to the lower index) with one barrier: every thread
// reduces the per-warp results itself.  The caller separates consecutive
// calls by at least one barrier.
__device__ int bargmax(float val, int idx, float* shv, int* shi) {
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_down_sync(0xffffffffu, val, o);
        int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { shv[wid] = val; shi[wid] = idx; }
    __syncthreads();
    float bv = shv[0];
    int bi = shi[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
        if (shv[i] > bv || (shv[i] == bv && shi[i] < bi)) { bv = shv[i]; bi = shi[i]; }
    return bi;
}

__global__ void __launch_bounds__(GT_MAX, 4) k_green32b(const float* __restrict__ Ypl, const double2* __restrict__ Tinv,
                                                   const double2* __restrict__ DR, float2* __restrict__ work,
                                                   float2* __restrict__ work2, float2* __restrict__ G,
                                                   const double* __restrict__ eps, double* __restrict__ ws,
                                                   int* __restrict__ status, int M, double lscale, double mu_T,
                                                   int constraint, Planes P, size_t wstride, double kdt) {
    extern __shared__ unsigned char smem_raw[];
    float2* Ps = reinterpret_cast<float2*>(smem_raw);        // [M][PSTR] panel / [M][NB] staged triangle block
    float2* Us = Ps + (size_t)M * PSTR;                        // [NB][M]  U12 rows; also the 32 x 33 tiles
    float2* drs = Us + us_len(M);                              // [M]
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
    __shared__ double lsum_s;
    __shared__ double2 ldm_s;
    __shared__ float2 rowp[NB], rowj[NB];
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
    // the two sums only thread 0 needs at the end are kept in shared memory,
    // not in registers held through the LU and the solves
    lsum = bsum(lsum, shd);
    if (tid == 0) {
        nswap = 0;
        lsum_s = lsum;
    }
    __syncthreads();
    {
        // 32 x 32 tiles: the chain planes are read along i (their contiguous
        // direction) into shared memory, T^-1 and Mt along j
        float2* tile = Us;                                       // [32][33] (TILE)
        const int lane = tid & 31, wid = tid >> 5, nwarp = GT >> 5;
        for (int ib = 0; ib < M; ib += 32)
            for (int jb = 0; jb < M; jb += 32) {
                for (int r = wid; r < 32; r += nwarp) {
                    const int i = ib + lane, j = jb + r;
                    tile[r * 33 + lane] = (i < M && j < M) ? P.load(Yw, i, j) : make_float2(0.f, 0.f);
                }
                __syncthreads();
                for (int r = wid; r < 32; r += nwarp) {
                    const int i = ib + r, j = jb + lane;
                    if (i < M && j < M) {
                        const long e = (long)i * M + j;
                        const double2 t = Tw[e] * ((double)dlb[i] * (double)drb[j]);
                        const float2 y = cmul(tile[lane * 33 + r], drs[j]) * dls[i];
                        A[e] = make_float2((float)t.x + y.x, (float)t.y + y.y);
                    }
                }
                __syncthreads();
            }
    }

    // ---------------------------------------------------------------- blocked LU
    for (int jb = 0; jb < M; jb += NB) {
        const int nb = min(NB, M - jb);
        const int rows = M - jb;
        for (int e = tid; e < rows * nb; e += GT) {
            const int r = e / nb, c = e % nb;
            Ps[r * PSTR + c] = A[(long)(jb + r) * M + jb + c];
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            float best = -1.0f;
            int bidx = M;
            for (int r = j + tid; r < rows; r += GT) {
                const float2 v = Ps[r * PSTR + j];
                const float a1 = fabsf(v.x) + fabsf(v.y);
                if (a1 > best) { best = a1; bidx = r; }
            }
            int p = bargmax(best, bidx, shv, shi);
            if (p >= rows) {
                p = j;
                if (tid == 0) atomicOr(status, 1);
            }
            // stash the pivot row and row j, then update every row from the
            // stash or from itself: no row is read after another thread wrote it
            for (int c = tid; c < nb; c += GT) {
                rowp[c] = Ps[p * PSTR + c];
                rowj[c] = Ps[j * PSTR + c];
            }
            __syncthreads();
            const float2 pv = rowp[j];
            const float n2 = pv.x * pv.x + pv.y * pv.y;
            const float2 ip = make_float2(pv.x / n2, -pv.y / n2);
            if (tid == 0) {
                if (!(n2 > 0.0f)) atomicOr(status, 1);
                piv[jb + j] = jb + p;
                invU[jb + j] = ip;
            }
            for (int c = tid; c < nb; c += GT) Ps[j * PSTR + c] = rowp[c];
            for (int r = j + 1 + tid; r < rows; r += GT) {
                float2* dst = Ps + r * PSTR;
                const float2* src = r == p ? rowj : dst;
                if (r == p)    // the swapped row keeps row j's earlier multipliers
                    for (int c = 0; c < j; ++c) dst[c] = rowj[c];
                const float2 l = cmul(src[j], ip);
                for (int c = j + 1; c < nb; ++c) dst[c] = csub_mul(src[c], l, rowp[c]);
                dst[j] = l;
            }
            __syncthreads();
        }
        for (int e = tid; e < rows * nb; e += GT) {
            const int r = e / nb, c = e % nb;
            A[(long)(jb + r) * M + jb + c] = Ps[r * PSTR + c];
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
        // U12 = L11^-1 A12, one column per thread.  Only a full panel has
        // columns to its right (a narrower one is the last, nb = M - jb), so
        // here and in the trailing update nb = NB.
        const int c0 = jb + nb;
        const int ncr = M - c0;
        for (int c = tid; c < ncr; c += GT) {
            float2 x[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) x[q] = A[(long)(jb + q) * M + c0 + c];
#pragma unroll
            for (int q = 1; q < NB; ++q) {
                float2 s = x[q];
#pragma unroll
                for (int q2 = 0; q2 < q; ++q2) s = csub_mul(s, Ps[q * PSTR + q2], x[q2]);
                x[q] = s;
            }
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                A[(long)(jb + q) * M + c0 + c] = x[q];
                Us[q * M + c] = x[q];
            }
        }
        __syncthreads();
        // A22 -= L21 U12 in TX x TY micro-tiles (rows and columns strided so
        // that a warp reads consecutive columns)
        const int nrr = M - c0;
        if (nrr > 0) {
            const int tr = (nrr + TX - 1) / TX, tc = (ncr + TY - 1) / TY;
            for (int t = tid; t < tr * tc; t += GT) {
                const int rg = t / tc, cg = t % tc;
                float2 acc[TX][TY];
#pragma unroll
                for (int x = 0; x < TX; ++x)
#pragma unroll
                    for (int y = 0; y < TY; ++y) {
                        const int r = rg + x * tr, c = cg + y * tc;
                        acc[x][y] = (r < nrr && c < ncr) ? A[(long)(c0 + r) * M + c0 + c] : make_float2(0.f, 0.f);
                    }
                // unguarded shared reads: a row r < nrr + TX - 1 of the panel
                // stays below row M + TX - 1 (the U12 region follows the
                // panel), a column c < ncr + TY - 1 stays inside row k of U12;
                // products of rows or columns past the edge are not stored
#pragma unroll 1
                for (int k = 0; k < NB; ++k) {
                    float2 a[TX], b[TY];
#pragma unroll
                    for (int x = 0; x < TX; ++x) a[x] = Ps[(NB + rg + x * tr) * PSTR + k];
#pragma unroll
                    for (int y = 0; y < TY; ++y) b[y] = Us[k * M + cg + y * tc];
#pragma unroll
                    for (int x = 0; x < TX; ++x)
#pragma unroll
                        for (int y = 0; y < TY; ++y) acc[x][y] = csub_mul(acc[x][y], a[x], b[y]);
                }
#pragma unroll
                for (int x = 0; x < TX; ++x)
#pragma unroll
                    for (int y = 0; y < TY; ++y) {
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
    if (tid == 0) ldm_s = ldm;

    // ---------------------------------------------------------------- X U = Y D_Rs
    for (int jb = 0; jb < M; jb += NB) {
        const int nb = min(NB, M - jb);
        for (int e = tid; e < (jb + nb) * NB; e += GT) {   // columns q >= nb zero-filled
            const int m = e / NB, q = e % NB;
            Ps[m * NB + q] = q < nb ? A[(long)m * M + jb + q] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int i = tid; i < M; i += GT) {
            float2 s[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
                s[q] = q < nb ? cmul(P.load(Yw, i, jb + q), drs[jb + q]) : make_float2(0.f, 0.f);
            for (int m = 0; m < jb; m += SU) {   // jb is a multiple of NB = SU
                float2 x[SU];
#pragma unroll
                for (int u = 0; u < SU; ++u) x[u] = X[(long)(m + u) * M + i];
#pragma unroll
                for (int q = 0; q < NB; ++q)      // no guard: columns q >= nb are zero
#pragma unroll
                    for (int u = 0; u < SU; ++u) s[q] = csub_mul(s[q], x[u], Ps[(m + u) * NB + q]);
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
                if (q < nb) X[(long)(jb + q) * M + i] = s[q];
        }
        __syncthreads();
    }
    // ---------------------------------------------------------------- W L = X (in place)
    const int nblk = (M + NB - 1) / NB;
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int jb = bi * NB;
        const int nb = min(NB, M - jb);
        for (int e = tid; e < (M - jb) * NB; e += GT) {   // columns q >= nb zero-filled
            const int m = jb + e / NB, q = e % NB;
            Ps[(m - jb) * NB + q] = q < nb ? A[(long)m * M + jb + q] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int i = tid; i < M; i += GT) {
            float2 s[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
                s[q] = q < nb ? X[(long)(jb + q) * M + i] : make_float2(0.f, 0.f);
            int m = jb + nb;
            for (; m + SU <= M; m += SU) {
                float2 x[SU];
#pragma unroll
                for (int u = 0; u < SU; ++u) x[u] = X[(long)(m + u) * M + i];
#pragma unroll
                for (int q = 0; q < NB; ++q)      // no guard: columns q >= nb are zero
#pragma unroll
                    for (int u = 0; u < SU; ++u) s[q] = csub_mul(s[q], x[u], Ps[(m + u - jb) * NB + q]);
            }
            for (; m < M; ++m) {
                const float2 x = X[(long)m * M + i];
#pragma unroll
                for (int q = 0; q < NB; ++q) s[q] = csub_mul(s[q], x, Ps[(m - jb) * NB + q]);
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
                if (q < nb) X[(long)(jb + q) * M + i] = s[q];
        }
        __syncthreads();
    }
    // G[i][c] = delta_ic - W[i][iperm[c]] dls[c], through 32 x 33 shared tiles
    // (reads of W columns and writes of G rows both contiguous)
    for (int m = tid; m < M; m += GT) piv[perm[m]] = m;       // piv <- inverse permutation
    __syncthreads();
    float2* tile = Us;                                           // [32][33] (TILE)
    const int lane = tid & 31, wid = tid >> 5, nwarp = GT >> 5;
    for (int ib = 0; ib < M; ib += 32)
        for (int cb = 0; cb < M; cb += 32) {
            for (int r = wid; r < 32; r += nwarp) {
                const int c = cb + r, i = ib + lane;
                tile[r * 33 + lane] = (c < M && i < M) ? X[(long)piv[c] * M + i] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int r = wid; r < 32; r += nwarp) {
                const int i = ib + r, c = cb + lane;
                if (i < M && c < M) {
                    float2 g = tile[lane * 33 + r] * (-dls[c]);
                    if (c == i) g.x += 1.0f;
                    Gw[(long)i * M + c] = g;
                }
            }
            __syncthreads();
        }
    __syncthreads();
    double2 trg = make_double2(0.0, 0.0);
    for (int i = tid; i < M; i += GT) {
        const float2 g = Gw[(long)i * M + i];
        trg = trg + make_double2(g.x, g.y);
    }
    trg = bsum(trg, shc);
    if (tid == 0)
        green_weight_tail(ws + (long)WSTRIDE * w, ldm_s, lsum_s, nswap, trg, M, kdt, constraint, status);
}

}  // namespace

size_t green32b_smem(int M) {
    return ((size_t)M * PSTR + us_len(M)) * sizeof(float2) + (size_t)M * (2 * sizeof(float2) + 3 * sizeof(float) + 2 * sizeof(int));
}

cudaError_t launch_green32b(ftq_ctx* c, int k, float2* G, double* ws) {
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
    const double lscale = left_scale(c, k);
    int nt = (M + 31) / 32 * 32;
    nt = nt < 256 ? 256 : (nt > GT_MAX ? GT_MAX : nt);
    LaunchScope ls(c, FTQ_K_GREEN);
    k_green32b<<<c->W, nt, sm, c->stream>>>(c->Ypl, c->Tinv, c->DR, c->w32, c->w2_32, G ? G : c->G32, c->tab.eps,
                                           ws ? ws : c->wstate,
                                           c->status, M, lscale, c->sys.mu_T, c->opts.constraint, P, 2 * P.part,
                                           (double)k * c->sys.dtau);
    return cudaGetLastError();
}

}  // namespace ftq

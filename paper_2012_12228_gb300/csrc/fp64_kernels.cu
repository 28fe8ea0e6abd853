// Complex128 kernels of the walker slice: force bias and HS fields, the
// Taylor-Horner application of B to the chain, Householder QRCP
// stabilisation, and the two-sided stable Green's function with ln det and
// the phaseless weight (the estimators are in estimators.cu).  One walker per thread block
// for the factorisations; tiled batched GEMM for the chain.
#include <cmath>

#include "block_reduce.cuh"
#include "complex_math.cuh"
#include "ftq_internal.h"

namespace ftq {
namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- init
__global__ void k_init_matrices(double2* Y, double2* Tinv, double2* G, const double* g0, int M, long total) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    int ij = (int)(e % ((long)M * M));
    int i = ij / M, j = ij % M;
    double2 one = make_double2(i == j ? 1.0 : 0.0, 0.0);
    Y[e] = one;
    Tinv[e] = one;
    G[e] = make_double2(i == j ? g0[i] : 0.0, 0.0);
}

__global__ void k_init_walkers(double2* DR, double* ws, int M, int W, double ld0) {
    int w = blockIdx.x;
    for (int i = threadIdx.x; i < M; i += blockDim.x) DR[(long)w * M + i] = make_double2(1.0, 0.0);
    if (threadIdx.x == 0) {
        double* s = ws + (long)WSTRIDE * w;
        for (int q = 0; q < WSTRIDE; ++q) s[q] = 0.0;
        s[2] = 1.0;
        s[3] = ld0;
        s[12] = (double)M;
    }
}

// ---------------------------------------------------------------- force bias
// rho_Q = sum_{(a,b): n_a - n_b = Q} P_ab with P = I - G^T, so for Q != 0
// rho_Q = -sum G[b][a].  <v_A> = 2 i c (rho_Q + rho_-Q), <v_B> = -2 c (rho_Q -
// rho_-Q); xbar = -sqrt(dtau) <v>; y = x - xbar; the V generator
// phi(+Q) = sqrt(dtau) c i (y_A + i y_B), phi(-Q) = sqrt(dtau) c i (y_A - i y_B).
__device__ __forceinline__ double2 to_c128(double2 v) { return v; }
__device__ __forceinline__ double2 to_c128(float2 v) { return make_double2(v.x, v.y); }

template <typename GT>
__global__ void k_force_bias(const GT* __restrict__ G, const double* __restrict__ x,
                             double2* __restrict__ phi, float2* __restrict__ phi32, double* __restrict__ ws,
                             const int* __restrict__ pptr, const int* __restrict__ pa,
                             const int* __restrict__ pb, const double* __restrict__ cq,
                             int M, int nqh, double sdt) {
    __shared__ double2 sh[32];
    const int w = blockIdx.x;
    const GT* Gw = G + (long)w * M * M;
    const double* xw = x + (long)w * 2 * nqh;
    double2* ph = phi + (long)w * (2 * nqh + 1);
    float2* ph32 = phi32 ? phi32 + (long)w * (2 * nqh + 1) : nullptr;
    double2 gauss = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        ph[0] = make_double2(0.0, 0.0);
        if (ph32) ph32[0] = make_float2(0.f, 0.f);
    }
    for (int q = threadIdx.x; q < nqh; q += blockDim.x) {
        double2 rp = make_double2(0.0, 0.0), rm = make_double2(0.0, 0.0);
        for (int e = pptr[1 + 2 * q]; e < pptr[2 + 2 * q]; ++e) rp = rp - to_c128(Gw[(long)pb[e] * M + pa[e]]);
        for (int e = pptr[2 + 2 * q]; e < pptr[3 + 2 * q]; ++e) rm = rm - to_c128(Gw[(long)pb[e] * M + pa[e]]);
        const double c = cq[q];
        double2 vA = times_i((rp + rm) * (2.0 * c));
        double2 vB = (rp - rm) * (-2.0 * c);
        double2 xbA = vA * (-sdt), xbB = vB * (-sdt);
        double xA = xw[2 * q], xB = xw[2 * q + 1];
        double2 yA = make_double2(xA - xbA.x, -xbA.y);
        double2 yB = make_double2(xB - xbB.x, -xbB.y);
        double2 iyB = times_i(yB);
        const double2 pp = times_i(yA + iyB) * (sdt * c), pm = times_i(yA - iyB) * (sdt * c);
        ph[1 + 2 * q] = pp;
        ph[2 + 2 * q] = pm;
        if (ph32) {
            ph32[1 + 2 * q] = make_float2((float)pp.x, (float)pp.y);
            ph32[2 + 2 * q] = make_float2((float)pm.x, (float)pm.y);
        }
        gauss = gauss + xbA * xA - cmul(xbA, xbA) * 0.5 + xbB * xB - cmul(xbB, xbB) * 0.5;
    }
    gauss = block_sum(gauss, sh);
    if (threadIdx.x == 0) {
        ws[(long)WSTRIDE * w + 5] = gauss.x;
        ws[(long)WSTRIDE * w + 6] = gauss.y;
    }
}

// ---------------------------------------------------------------- chain GEMM
// out[i][c] = os_i (us_i Yu[i][c] + alpha sum_k V[i][k] zs_k Zin[k][c]),
// V[i][k] = phi[vidx[i][k]]: one Horner step of exp(V) applied to the chain.
constexpr int CT = 32;   // output tile
constexpr int CK = 16;   // k tile

__global__ void __launch_bounds__(256) k_chain_step(const double2* __restrict__ Zin, const double2* __restrict__ Yu,
                                                   double2* __restrict__ out, const double2* __restrict__ phi,
                                                   const uint16_t* __restrict__ vidx, const double* __restrict__ zs,
                                                   const double* __restrict__ us, const double* __restrict__ os,
                                                   double alpha, int M, int nslot, int tiles,
                                                   const double* __restrict__ rank_ws) {
    __shared__ double2 As[CK][CT + 1];
    __shared__ double2 Bs[CK][CT + 1];
    const int w = blockIdx.y;
    const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles;
    const int r0 = ti * CT, c0 = tj * CT;
    // low rank: only the first m columns of the chain are live
    if (rank_ws && c0 >= (int)rank_ws[(long)WSTRIDE * w + 12]) return;
    const long off = (long)w * M * M;
    const double2* Z = Zin + off;
    const double2* ph = phi + (long)w * nslot;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double2 acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < M; k0 += CK) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            int e = threadIdx.x + 256 * l;        // 0..511
            int r = e >> 4, kk = e & 15;          // A tile: 32 rows x 16 k
            int i = r0 + r, k = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (i < M && k < M) v = ph[vidx[(long)i * M + k]];
            As[kk][r] = v;
            int kb = e >> 5, cb = e & 31;         // B tile: 16 k x 32 cols
            int kr = k0 + kb, cc = c0 + cb;
            double2 z = make_double2(0.0, 0.0);
            if (kr < M && cc < M) {
                z = Z[(long)kr * M + cc];
                if (zs) z = z * zs[kr];
            }
            Bs[kb][cb] = z;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CK; ++kk) {
            double2 a0 = As[kk][ty], a1 = As[kk][ty + 16];
            double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = cfma(a0, b0, acc[0][0]);
            acc[0][1] = cfma(a0, b1, acc[0][1]);
            acc[1][0] = cfma(a1, b0, acc[1][0]);
            acc[1][1] = cfma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int i = r0 + ty + 16 * a, c = c0 + tx + 16 * b;
            if (i < M && c < M) {
                long e = off + (long)i * M + c;
                double2 v = Yu[e] * us[i] + acc[a][b] * alpha;
                if (os) v = v * os[i];
                out[e] = v;
            }
        }
}

// ---------------------------------------------------------------- QRCP
// Householder QR with column pivoting of C = Y diag(D_R) (Businger-Golub:
// pivot = remaining column of largest norm, ties to the lowest index).
// Reflector H = I - tau u u^H with u = x - beta e_1, beta = -e^{i arg x_0}|x|,
// so H x = beta e_1 and R_jj = beta.  Outputs: Q (next chain start), D_R =
// diag R, T^-1 <- T^-1 Pi^T (D^-1 R)^-1, parity of Pi.
__global__ void k_qrcp(const double2* __restrict__ Yin, double2* __restrict__ Qout,
                       double2* __restrict__ work, double2* __restrict__ work2,
                       double2* __restrict__ DR, double2* __restrict__ Tinv,
                       double2* __restrict__ hh, double* __restrict__ htau,
                       double* __restrict__ ws, int* __restrict__ status, int M) {
    extern __shared__ unsigned char smem_raw[];
    double* cn = reinterpret_cast<double*>(smem_raw);          // column norms [M]
    int* perm = reinterpret_cast<int*>(cn + M);                 // [M]
    __shared__ double shv[32];
    __shared__ int shi[32];
    __shared__ int nswap;
    const int w = blockIdx.x;
    const long off = (long)w * M * M;
    double2* C = work + off;
    double2* Q = Qout + off;
    double2* XT = work2 + off;
    double2* Ti = Tinv + off;
    const double2* Yw = Yin + off;
    double2* u0 = hh + (long)w * M;
    double* tau = htau + (long)w * M;
    const int nt = blockDim.x;

    for (long e = threadIdx.x; e < (long)M * M; e += nt) {
        int c = (int)(e % M);
        C[e] = cmul(Yw[e], DR[(long)w * M + c]);
    }
    for (int c = threadIdx.x; c < M; c += nt) perm[c] = c;
    if (threadIdx.x == 0) nswap = 0;
    __syncthreads();

    for (int j = 0; j < M; ++j) {
        double best = -1.0;
        int bidx = M;
        for (int c = j + threadIdx.x; c < M; c += nt) {
            double s = 0.0;
            for (int r = j; r < M; ++r) s += abs2(C[(long)r * M + c]);
            cn[c] = s;
            if (s > best) { best = s; bidx = c; }
        }
        int pc = block_argmax(best, bidx, shv, shi);
        if (pc >= M) {                       // every candidate norm was NaN
            pc = j;
            if (threadIdx.x == 0) atomicOr(status, 1);
        }
        if (pc != j) {
            for (int r = threadIdx.x; r < M; r += nt) {
                double2 t = C[(long)r * M + j];
                C[(long)r * M + j] = C[(long)r * M + pc];
                C[(long)r * M + pc] = t;
            }
            if (threadIdx.x == 0) {
                int t = perm[j]; perm[j] = perm[pc]; perm[pc] = t;
                double tn = cn[j]; cn[j] = cn[pc]; cn[pc] = tn;
                nswap ^= 1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double2 al = C[(long)j * M + j];
            double sig = sqrt(cn[j]);
            double aa = sqrt(abs2(al));
            double2 beta = aa > 0.0 ? al * (-sig / aa) : make_double2(-sig, 0.0);
            double uhu = 2.0 * sig * (sig + aa);
            u0[j] = al - beta;
            tau[j] = uhu > 0.0 ? 2.0 / uhu : 0.0;
            C[(long)j * M + j] = beta;
            if (!(sig > 0.0)) atomicOr(status, 1);
        }
        __syncthreads();
        const double2 uj = u0[j];
        const double tj = tau[j];
        for (int c = j + 1 + threadIdx.x; c < M; c += nt) {
            double2 s = cmul(conj(uj), C[(long)j * M + c]);
            for (int r = j + 1; r < M; ++r) s = cfma(conj(C[(long)r * M + j]), C[(long)r * M + c], s);
            s = s * tj;
            C[(long)j * M + c] = cfms(uj, s, C[(long)j * M + c]);
            for (int r = j + 1; r < M; ++r) C[(long)r * M + c] = cfms(C[(long)r * M + j], s, C[(long)r * M + c]);
        }
        __syncthreads();
    }
    // Q = H_0 H_1 ... H_{M-1} by backward accumulation
    for (long e = threadIdx.x; e < (long)M * M; e += nt) {
        int i = (int)(e / M), c = (int)(e % M);
        Q[e] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int j = M - 1; j >= 0; --j) {
        const double2 uj = u0[j];
        const double tj = tau[j];
        for (int c = j + threadIdx.x; c < M; c += nt) {
            double2 s = cmul(conj(uj), Q[(long)j * M + c]);
            for (int r = j + 1; r < M; ++r) s = cfma(conj(C[(long)r * M + j]), Q[(long)r * M + c], s);
            s = s * tj;
            Q[(long)j * M + c] = cfms(uj, s, Q[(long)j * M + c]);
            for (int r = j + 1; r < M; ++r) Q[(long)r * M + c] = cfms(C[(long)r * M + j], s, Q[(long)r * M + c]);
        }
        __syncthreads();
    }
    // D = diag R; U = D^-1 R (strict upper part scaled in place)
    for (int j = threadIdx.x; j < M; j += nt) DR[(long)w * M + j] = C[(long)j * M + j];
    for (long e = threadIdx.x; e < (long)M * M; e += nt) {
        int i = (int)(e / M), c = (int)(e % M);
        if (c > i) C[e] = cdiv(C[e], C[(long)i * M + i]);
    }
    __syncthreads();
    // T^-1 <- T^-1[:, perm] U^-1, one row per thread (XT column-major)
    for (int i = threadIdx.x; i < M; i += nt) {
        for (int j = 0; j < M; ++j) {
            double2 s = Ti[(long)i * M + perm[j]];
            for (int m = 0; m < j; ++m) s = cfms(XT[(long)m * M + i], C[(long)m * M + j], s);
            XT[(long)j * M + i] = s;
        }
        for (int j = 0; j < M; ++j) Ti[(long)i * M + j] = XT[(long)j * M + i];
    }
    if (threadIdx.x == 0) {
        double* s = ws + (long)WSTRIDE * w;
        s[7] = (double)(((int)s[7]) ^ nswap);
    }
}

// ---------------------------------------------------------------- Green's function
// G(tau_k) = (I + R D_L)^-1 with R = Y D_R T, D_L = B_T^(n-k):
//   Mt = D_Lb T^-1 D_Rb + D_Ls Y D_Rs,  G = I - Y D_Rs Mt^-1 D_Ls,
//   ln det(I + A) = -sum ln D_Lb - sum ln D_Rb + ln det Mt + ln det T,
// then ln S_k = 2 (ln det_k - ln det_{k-1}) and the weight (Eqs. import,
// phimport, theta).
__global__ void k_green(const double2* __restrict__ Y, const double2* __restrict__ Tinv,
                        const double2* __restrict__ DR, double2* __restrict__ work,
                        double2* __restrict__ work2, double2* __restrict__ G,
                        const double* __restrict__ eps, double* __restrict__ ws,
                        int* __restrict__ status, int M, double lscale, double mu_T,
                        int constraint, int update, int with_gauss, double kdt) {
    extern __shared__ unsigned char smem_raw[];
    double2* drs = reinterpret_cast<double2*>(smem_raw);     // [M]
    double2* invU = drs + M;                                 // [M]
    double* dls = reinterpret_cast<double*>(invU + M);       // [M]
    double* dlb = dls + M;                                   // [M]
    double* drb = dlb + M;                                   // [M]
    int* perm = reinterpret_cast<int*>(drb + M);             // [M]
    __shared__ double shv[32];
    __shared__ int shi[32];
    __shared__ double2 shc[32];
    __shared__ int nswap;
    const int w = blockIdx.x;
    const long off = (long)w * M * M;
    const int nt = blockDim.x;
    double2* A = work + off;
    double2* XT = work2 + off;
    const double2* Yw = Y + off;
    const double2* Tw = Tinv + off;
    double2* Gw = G + off;

    double lsum = 0.0;
    for (int i = threadIdx.x; i < M; i += nt) {
        double dl = exp(-lscale * (eps[i] - mu_T));
        if (dl > 1.0) { dlb[i] = 1.0 / dl; dls[i] = 1.0; } else { dlb[i] = 1.0; dls[i] = dl; }
        double2 d = DR[(long)w * M + i];
        double a = sqrt(abs2(d));
        if (a > 1.0) { drb[i] = 1.0 / a; drs[i] = d * (1.0 / a); } else { drb[i] = 1.0; drs[i] = d; }
        lsum += log(dlb[i]) + log(drb[i]);
        perm[i] = i;
    }
    if (threadIdx.x == 0) nswap = 0;
    __syncthreads();
    for (long e = threadIdx.x; e < (long)M * M; e += nt) {
        int i = (int)(e / M), j = (int)(e % M);
        A[e] = Tw[e] * (dlb[i] * drb[j]) + cmul(Yw[e], drs[j]) * dls[i];
    }
    __syncthreads();
    // LU with partial pivoting, in place
    for (int j = 0; j < M; ++j) {
        double best = -1.0;
        int bidx = M;
        for (int i = j + threadIdx.x; i < M; i += nt) {
            double v = abs1(A[(long)i * M + j]);
            if (v > best) { best = v; bidx = i; }
        }
        int p = block_argmax(best, bidx, shv, shi);
        if (p >= M) {                        // every candidate pivot was NaN
            p = j;
            if (threadIdx.x == 0) atomicOr(status, 1);
        }
        if (p != j) {
            for (int c = threadIdx.x; c < M; c += nt) {
                double2 t = A[(long)j * M + c];
                A[(long)j * M + c] = A[(long)p * M + c];
                A[(long)p * M + c] = t;
            }
            if (threadIdx.x == 0) {
                int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
                nswap ^= 1;
            }
        }
        __syncthreads();
        const double2 piv = A[(long)j * M + j];
        if (!(abs2(piv) > 0.0)) {
            if (threadIdx.x == 0) atomicOr(status, 1);
        }
        const double2 ip = cinv(piv);
        for (int i = j + 1 + threadIdx.x; i < M; i += nt) A[(long)i * M + j] = cmul(A[(long)i * M + j], ip);
        if (threadIdx.x == 0) invU[j] = ip;
        __syncthreads();
        for (int c = j + 1 + threadIdx.x; c < M; c += nt) {
            const double2 u = A[(long)j * M + c];
            for (int i = j + 1; i < M; ++i) A[(long)i * M + c] = cfms(A[(long)i * M + j], u, A[(long)i * M + c]);
        }
        __syncthreads();
    }
    // ln det Mt = sum ln U_jj + i pi (row-swap parity)
    double2 ldm = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < M; j += nt) ldm = ldm + clog(A[(long)j * M + j]);
    ldm = block_sum(ldm, shc);
    lsum = block_sum(lsum, shv);
    // X = (Y D_Rs) U^-1 L^-1 solved row by row (XT column-major), then
    // G[i][perm[m]] = delta - X[i][m] dls[perm[m]].
    for (int i = threadIdx.x; i < M; i += nt) {
        for (int j = 0; j < M; ++j) {
            double2 s = cmul(Yw[(long)i * M + j], drs[j]);
            for (int m = 0; m < j; ++m) s = cfms(XT[(long)m * M + i], A[(long)m * M + j], s);
            XT[(long)j * M + i] = cmul(s, invU[j]);
        }
        for (int j = M - 2; j >= 0; --j) {
            double2 s = XT[(long)j * M + i];
            for (int m = j + 1; m < M; ++m) s = cfms(XT[(long)m * M + i], A[(long)m * M + j], s);
            XT[(long)j * M + i] = s;
        }
        for (int m = 0; m < M; ++m) {
            int c = perm[m];
            double2 g = XT[(long)m * M + i] * (-dls[c]);
            if (c == i) g.x += 1.0;
            Gw[(long)i * M + c] = g;
        }
    }
    __syncthreads();
    double2 trg = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < M; i += nt) trg = trg + Gw[(long)i * M + i];
    trg = block_sum(trg, shc);
    if (threadIdx.x == 0) {
        double* s = ws + (long)WSTRIDE * w;
        double2 ld = ldm;
        ld.x -= lsum;
        ld.y += kPi * (double)(nswap ^ ((int)s[7]));
        if (!isfinite(ld.x) || !isfinite(ld.y)) atomicOr(status, 1);
        // d ln det(I + A_k)/dmu = k dtau (M - tr G(tau_k)): every B carries exp(dtau mu)
        const double2 tk = make_double2(kdt * ((double)M - trg.x), -kdt * trg.y);
        if (update) {
            double2 lnS = make_double2(2.0 * (ld.x - s[3]), 2.0 * (ld.y - s[4]));
            const double2 dlnS = make_double2(2.0 * (tk.x - s[9]), 2.0 * (tk.y - s[10]));
            const double gr = with_gauss ? s[5] : 0.0, gi = with_gauss ? s[6] : 0.0;
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

}  // namespace

cudaError_t launch_init_walkers(ftq_ctx* c) {
    const int M = c->M, W = c->W;
    double ld0 = 0.0;
    for (int i = 0; i < M; ++i) ld0 += std::log1p(std::exp(-c->sys.beta * (c->sys.eps[i] - c->sys.mu_T)));
    long total = (long)W * M * M;
    LaunchScope ls0(c, FTQ_K_INIT);
    k_init_matrices<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(c->Y ? c->Y : c->zbuf[1], c->Tinv, c->G,
                                                                           c->tab.g0, M, total);
    c->launches[FTQ_K_INIT] += 1;
    k_init_walkers<<<W, 64, 0, c->stream>>>(c->DR, c->wstate, M, W, ld0);
    c->k = 0;
    c->g64_valid = true;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c->opts.precision != FTQ_FP64) e = mixed_init(c);
    return e;
}

cudaError_t launch_force_bias_any(ftq_ctx* c, const double* x, const void* G, bool g32) {
    LaunchScope ls(c, FTQ_K_FORCE_BIAS);
    if (g32)
        k_force_bias<float2><<<c->W, 256, 0, c->stream>>>(reinterpret_cast<const float2*>(G), x, c->phi, c->phi32,
                                                          c->wstate,
                                                          c->tab.pair_ptr, c->tab.pair_a, c->tab.pair_b, c->tab.cq,
                                                          c->M, c->sys.nq_half, std::sqrt(c->sys.dtau));
    else
        k_force_bias<double2><<<c->W, 256, 0, c->stream>>>(reinterpret_cast<const double2*>(G), x, c->phi,
                                                           c->phi32, c->wstate, c->tab.pair_ptr, c->tab.pair_a, c->tab.pair_b,
                                                           c->tab.cq, c->M, c->sys.nq_half, std::sqrt(c->sys.dtau));
    return cudaGetLastError();
}

cudaError_t launch_force_bias(ftq_ctx* c, const double* x) {
    if (c->opts.precision != FTQ_FP64 && !c->g64_valid) return launch_force_bias_any(c, x, c->G32, true);
    return launch_force_bias_any(c, x, c->G, false);
}

cudaError_t launch_chain(ftq_ctx* c) {
    if (c->opts.precision != FTQ_FP64) return mixed_chain(c);
    const int M = c->M, p = c->opts.exp_order;
    const int tiles = (M + CT - 1) / CT;
    dim3 grid(tiles * tiles, c->W);
    // Horner: Z_p = h Y + V h Y / p;  Z_j = h Y + V Z_{j+1} / j;  Y' = h Z_1
    const double2* zin = c->Y;
    int cur = 0;
    for (int j = p; j >= 1; --j) {
        double2* out = c->zbuf[cur];
        LaunchScope ls(c, FTQ_K_CHAIN);
        k_chain_step<<<grid, 256, 0, c->stream>>>(zin, c->Y, out, c->phi, c->tab.vidx,
                                                  j == p ? c->tab.h : nullptr, c->tab.h,
                                                  j == 1 ? c->tab.h : nullptr, 1.0 / j, M, c->nslot, tiles,
                                                  c->opts.low_rank_threshold > 0.0 ? c->wstate : nullptr);
        zin = out;
        cur ^= 1;
    }
    // the result sits in zbuf[cur ^ 1]; make it the chain
    double2* res = c->zbuf[cur ^ 1];
    c->zbuf[cur ^ 1] = c->Y;
    c->Y = res;
    return cudaGetLastError();
}

cudaError_t launch_qrcp64(ftq_ctx* c, const double2* Yin, double2* Qout) {
    const int M = c->M;
    size_t sm = sizeof(double) * M + sizeof(int) * M;
    int nt = fact_threads(M);
    LaunchScope ls(c, FTQ_K_QRCP);
    k_qrcp<<<c->W, nt, sm, c->stream>>>(Yin, Qout, c->work, c->work2, c->DR, c->Tinv, c->hh, c->htau,
                                       c->wstate, c->status, M);
    return cudaGetLastError();
}

cudaError_t launch_qrcp(ftq_ctx* c) {
    if (c->opts.precision != FTQ_FP64) return mixed_qrcp(c);
    if (c->opts.low_rank_threshold > 0.0) return launch_qrcp_lr(c);
    cudaError_t e = launch_qrcp64(c, c->Y, c->zbuf[0]);
    double2* q = c->zbuf[0];
    c->zbuf[0] = c->Y;
    c->Y = q;
    return e;
}

double left_scale(const ftq_ctx* c, int k) {
    const int power = c->opts.overlap == FTQ_OVERLAP_MODIFIED ? c->sys.n_slices : c->sys.n_slices - k;
    return (double)power * c->sys.dtau;
}

cudaError_t launch_green64(ftq_ctx* c, const double2* Y, int k, bool update, bool physical) {
    const int M = c->M;
    size_t sm = (2 * sizeof(double2) + 3 * sizeof(double) + sizeof(int)) * M;
    int nt = fact_threads(M);
    if (c->opts.low_rank_threshold > 0.0) return launch_green_lr(c, Y, k, update, physical);
    const double lscale = physical ? 0.0 : left_scale(c, k);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_green, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    LaunchScope ls(c, FTQ_K_GREEN);
    k_green<<<c->W, nt, sm, c->stream>>>(Y, c->Tinv, c->DR, c->work, c->work2, c->G, c->tab.eps, c->wstate,
                                        c->status, M, lscale, c->sys.mu_T, c->opts.constraint, update ? 1 : 0,
                                        physical ? 0 : 1, (double)k * c->sys.dtau);
    return cudaGetLastError();
}

cudaError_t launch_green(ftq_ctx* c, int k, bool update) {
    if (c->opts.precision != FTQ_FP64) return mixed_green(c, k);
    cudaError_t e = launch_green64(c, c->Y, k, update);
    // the modified overlap ends with the physical G(beta) and the ratio r
    if (e == cudaSuccess && k == c->sys.n_slices && c->opts.overlap == FTQ_OVERLAP_MODIFIED)
        e = launch_green64(c, c->Y, k, update, true);
    return e;
}

cudaError_t launch_copy_green(ftq_ctx* c, double2* out) {
    if (!c->g64_valid) {
        cudaError_t e0 = mixed_sync_g64(c);
        if (e0 != cudaSuccess) return e0;
    }
    return cudaMemcpyAsync(out, c->G, sizeof(double2) * (size_t)c->W * c->M * c->M, cudaMemcpyDeviceToDevice,
                           c->stream);
}

}  // namespace ftq

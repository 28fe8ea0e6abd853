// Stabilisation of the mixed-precision chain with pre-pivoting.
//
// The right block is A_R = Y D_R T with Y = (B's since the last QR) Q_R in
// FP32 and D_R, T^-1 in FP64.  Instead of pivoting at every Householder
// step, the columns of C = Y D_R are sorted once by their norms (the
// pre-pivoting of the GPU stratification work the paper cites for its
// stabilisation): C Pi has decreasing column norms, Y is well conditioned
// (a few B's times a unitary matrix) and the grading sits in D_R, so an
// unpivoted Householder QR of C Pi separates the scales like QRCP does.
//
//   k_qr_prepiv64 (FP64, one block per walker): norms, sort, C Pi, Householder
//       QR, D <- diag R, U = D^-1 R, T^-1 <- T^-1 Pi^T U^-1, permutation parity;
//       the reflectors are also written in FP32, one reflector per row.
//   k_form_q32 (FP32, one block per walker and 32-column panel): Q = H_0 ...
//       H_{M-1} applied to the identity panel in shared memory, written into
//       the chain planes as the new Y.
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"
#include "mixed_common.cuh"

namespace ftq {
namespace {

constexpr int QP = 32;   // columns per Q panel
constexpr int NBJ = 2;   // columns per block of the T^-1 update

__device__ double bsum_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = sh[0];
        for (int i = 1; i < (int)((blockDim.x + 31) >> 5); ++i) acc += sh[i];
        sh[0] = acc;
    }
    __syncthreads();
    double r = sh[0];
    __syncthreads();
    return r;
}

// (launch bounds: four 288-thread blocks per SM; measured faster than three
// uncapped blocks or smaller blocks at M = 257)
// Block sum of a complex value; every thread returns the total.
__device__ double2 bsum_c(double2 v, double2* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double2 acc = sh[0];
    for (int i = 1; i < (int)((blockDim.x + 31) >> 5); ++i) acc = acc + sh[i];
    __syncthreads();
    return acc;
}

// Householder reflector of column j from its squared norm s (rows >= j):
// beta = -|x| x_j/|x_j| replaces C[j][j]; u_j = x_j - beta, tau = 2/(u^H u).
__device__ void reflector_head(double2* C, double* htau_w, int* status, int M, int j, double s, double2* u0,
                               double* tau) {
    const double2 al = C[(long)j * M + j];
    const double sig = sqrt(s);
    const double aa = sqrt(abs2(al));
    const double2 beta = aa > 0.0 ? al * (-sig / aa) : make_double2(-sig, 0.0);
    const double uhu = 2.0 * sig * (sig + aa);
    *u0 = al - beta;
    *tau = uhu > 0.0 ? 2.0 / uhu : 0.0;
    htau_w[j] = *tau;
    C[(long)j * M + j] = beta;
    if (!(sig > 0.0)) atomicOr(status, 1);
}

__global__ void __launch_bounds__(288, 4) k_qr_prepiv64(const float* __restrict__ Ypl, double2* __restrict__ work,
                              double2* __restrict__ work2, double2* __restrict__ DR, double2* __restrict__ Tinv,
                              float2* __restrict__ VT, double* __restrict__ htau, double* __restrict__ xsum,
                              double* __restrict__ ws,
                              int* __restrict__ status, int M, Planes P, size_t wstride) {
    extern __shared__ unsigned char smem_raw[];
    double* ub = reinterpret_cast<double*>(smem_raw);      // [M][NBJ][3] U block of the T^-1 update
    double* cn = ub + 3 * NBJ * M;                         // [M] column norms of C
    int* perm = reinterpret_cast<int*>(cn + M);            // [M] C Pi column j = C column perm[j]
    unsigned char* seen = reinterpret_cast<unsigned char*>(perm + M);   // [M]
    __shared__ double shd[32];
    __shared__ double2 piv_u0, piv_u1, shc2[32];
    __shared__ double piv_tau, piv_tau1;
    __shared__ int parity;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w = blockIdx.x;
    const long off = (long)w * M * M;
    double2* C = work + off;
    double2* XT = work2 + off;
    double2* Ti = Tinv + off;
    double2* Dw = DR + (long)w * M;
    float2* V = VT + off;
    const float* Yw = Ypl + wstride * w;

    // column norms of C = Y D_R, then the rank of every column (descending
    // norm, ties to the lower index)
    for (int c = tid; c < M; c += nt) {
        double s = 0.0;
        for (int i = 0; i < M; ++i) {
            float2 y = P.load(Yw, i, c);
            s += (double)y.x * y.x + (double)y.y * y.y;
        }
        double v = s * abs2(Dw[c]);
        // a NaN norm would compare false both ways and give two columns one
        // rank (leaving an entry of perm unset); rank it last and latch
        if (v != v) {
            v = -INFINITY;
            atomicOr(status, 1);
        }
        cn[c] = v;
    }
    __syncthreads();
    for (int c = tid; c < M; c += nt) {
        int rank = 0;
        const double v = cn[c];
        for (int c2 = 0; c2 < M; ++c2) rank += (cn[c2] > v || (cn[c2] == v && c2 < c)) ? 1 : 0;
        perm[rank] = c;
        seen[c] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        // parity of the permutation = (M - number of cycles) mod 2
        int cycles = 0;
        for (int c = 0; c < M; ++c) {
            if (seen[c]) continue;
            ++cycles;
            for (int x = c; !seen[x]; x = perm[x]) seen[x] = 1;
        }
        parity = (M - cycles) & 1;
    }
    for (long e = tid; e < (long)M * M; e += nt) {
        const int i = (int)(e / M), j = (int)(e % M);
        const int src = perm[j];
        const float2 y = P.load(Yw, i, src);
        C[e] = cmul(make_double2(y.x, y.y), Dw[src]);
    }
    __syncthreads();

    // Householder QR of C Pi, two reflectors per pass over the trailing
    // columns: H_j is applied to column j + 1 first and u_{j+1} formed; then
    // every later column x takes both in one read pass (d1 = u_j^H x,
    // d2 = u_{j+1}^H x) and one write pass, x -= a1 u_j + a2 u_{j+1} with
    // a1 = tau_j d1 and a2 = tau_{j+1} (d2 - a1 u_{j+1}^H u_j).
    for (int j = 0; j < M; j += 2) {
        double s = 0.0;
        for (int r = j + tid; r < M; r += nt) s += abs2(C[(long)r * M + j]);
        s = bsum_d(s, shd);
        if (tid == 0) reflector_head(C, htau + (long)w * M, status, M, j, s, &piv_u0, &piv_tau);
        __syncthreads();
        const double2 uj = piv_u0;           // u_j[j]; u_j[r] = C[r][j] below
        const double tj = piv_tau;
        // reflector j in FP32 for the Q panels: V[j][r] = u_r, r >= j
        for (int r = j + tid; r < M; r += nt) {
            const double2 u = r == j ? uj : C[(long)r * M + j];
            V[(long)j * M + r] = make_float2((float)u.x, (float)u.y);
        }
        if (j + 1 >= M) break;
        // H_j on column j + 1
        double2 d = make_double2(0.0, 0.0);
        for (int r = j + tid; r < M; r += nt) {
            const double2 u = r == j ? uj : C[(long)r * M + j];
            d = cfma(conj(u), C[(long)r * M + j + 1], d);
        }
        const double2 a = bsum_c(d, shc2) * tj;
        for (int r = j + tid; r < M; r += nt) {
            const double2 u = r == j ? uj : C[(long)r * M + j];
            C[(long)r * M + j + 1] = cfms(u, a, C[(long)r * M + j + 1]);
        }
        __syncthreads();
        // reflector j + 1
        s = 0.0;
        for (int r = j + 1 + tid; r < M; r += nt) s += abs2(C[(long)r * M + j + 1]);
        s = bsum_d(s, shd);
        if (tid == 0) reflector_head(C, htau + (long)w * M, status, M, j + 1, s, &piv_u1, &piv_tau1);
        __syncthreads();
        const double2 u1 = piv_u1;           // u_{j+1}[j+1]; u_{j+1}[r] = C[r][j+1] below
        const double t1 = piv_tau1;
        for (int r = j + 1 + tid; r < M; r += nt) {
            const double2 u = r == j + 1 ? u1 : C[(long)r * M + j + 1];
            V[(long)(j + 1) * M + r] = make_float2((float)u.x, (float)u.y);
        }
        // g = u_{j+1}^H u_j (rows >= j + 1)
        double2 gp = make_double2(0.0, 0.0);
        for (int r = j + 1 + tid; r < M; r += nt) {
            const double2 u = r == j + 1 ? u1 : C[(long)r * M + j + 1];
            gp = cfma(conj(u), C[(long)r * M + j], gp);
        }
        const double2 g = bsum_c(gp, shc2);
        const double2 uj1 = C[(long)(j + 1) * M + j];    // u_j[j+1]
        for (int c = j + 2 + tid; c < M; c += nt) {
            const double2 x0 = C[(long)j * M + c], x1 = C[(long)(j + 1) * M + c];
            double2 d1 = cfma(conj(uj1), x1, cmul(conj(uj), x0));
            double2 d2 = cmul(conj(u1), x1);
            for (int r = j + 2; r < M; ++r) {
                const double2 x = C[(long)r * M + c];
                d1 = cfma(conj(C[(long)r * M + j]), x, d1);
                d2 = cfma(conj(C[(long)r * M + j + 1]), x, d2);
            }
            const double2 a1 = d1 * tj;
            const double2 a2 = cfms(a1, g, d2) * t1;
            C[(long)j * M + c] = cfms(uj, a1, x0);
            C[(long)(j + 1) * M + c] = cfms(u1, a2, cfms(uj1, a1, x1));
            for (int r = j + 2; r < M; ++r) {
                double2 x = C[(long)r * M + c];
                x = cfms(C[(long)r * M + j], a1, x);
                x = cfms(C[(long)r * M + j + 1], a2, x);
                C[(long)r * M + c] = x;
            }
        }
        __syncthreads();
    }
    for (int j = tid; j < M; j += nt) Dw[j] = C[(long)j * M + j];
    __syncthreads();
    for (long e = tid; e < (long)M * M; e += nt) {
        const int i = (int)(e / M), c = (int)(e % M);
        if (c > i) C[e] = cdiv(C[e], C[(long)i * M + i]);
    }
    __syncthreads();
    // Re U + Im U of the strict upper triangle, kept in the real parts of the
    // (no longer needed) lower triangle: U[m][j] -> C[j][m].x
    for (long e = tid; e < (long)M * M; e += nt) {
        const int j = (int)(e / M), m = (int)(e % M);
        if (m < j) {
            const double2 u = C[(long)m * M + j];
            C[e].x = u.x + u.y;
        }
    }
    __syncthreads();
    // T^-1 <- T^-1[:, perm] U^-1, one row per thread (XT column-major), in
    // blocks of NBJ columns: the block's entries of U (Re, Im and Re + Im) for
    // every earlier row m are staged in shared memory, so that each X[i][m]
    // read from memory serves NBJ columns.  The complex sums over m use three
    // real products per term (sum ac, sum bd, sum (a + b)(c + d): the
    // three-multiplication complex product), with a + b of X kept beside X
    // and c + d of U precomputed above; every column sums m = 0 .. j - 1 in
    // order, as the column-by-column solve does.
    double* XS = xsum + off;
    for (int jb = 0; jb < M; jb += NBJ) {
        const int nb = min(NBJ, M - jb);
        for (int e = tid; e < (jb + nb) * NBJ; e += nt) {
            const int m = e / NBJ, q = e % NBJ, j = jb + q;
            double ur = 0.0, ui = 0.0, us = 0.0;
            if (q < nb && m < j) {
                const double2 u = C[(long)m * M + j];
                ur = u.x;
                ui = u.y;
                us = C[(long)j * M + m].x;
            }
            ub[3 * e] = ur;
            ub[3 * e + 1] = ui;
            ub[3 * e + 2] = us;
        }
        __syncthreads();
        for (int i = tid; i < M; i += nt) {
            double pr[NBJ], qr[NBJ], rr[NBJ];
#pragma unroll
            for (int q = 0; q < NBJ; ++q) pr[q] = qr[q] = rr[q] = 0.0;
            for (int m = 0; m < jb; ++m) {
                const double2 x = XT[(long)m * M + i];
                const double xs = XS[(long)m * M + i];
                const double* u = ub + 3 * NBJ * m;
#pragma unroll
                for (int q = 0; q < NBJ; ++q) {
                    pr[q] = fma(x.x, u[3 * q], pr[q]);
                    qr[q] = fma(x.y, u[3 * q + 1], qr[q]);
                    rr[q] = fma(xs, u[3 * q + 2], rr[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < NBJ; ++q) {
                if (q < nb) {
                    const int j = jb + q;
                    for (int q2 = 0; q2 < q; ++q2) {          // m = jb + q2, solved above
                        const long o = (long)(jb + q2) * M + i;
                        const double2 x = XT[o];
                        const double* u = ub + 3 * (NBJ * (jb + q2) + q);
                        pr[q] = fma(x.x, u[0], pr[q]);
                        qr[q] = fma(x.y, u[1], qr[q]);
                        rr[q] = fma(XS[o], u[2], rr[q]);
                    }
                    double2 s = Ti[(long)i * M + perm[j]];
                    s.x -= pr[q] - qr[q];
                    s.y -= rr[q] - pr[q] - qr[q];
                    XT[(long)j * M + i] = s;
                    XS[(long)j * M + i] = s.x + s.y;
                }
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < M; i += nt)
        for (int j = 0; j < M; ++j) Ti[(long)i * M + j] = XT[(long)j * M + i];
    if (tid == 0) {
        double* st = ws + (long)WSTRIDE * w;
        st[7] = (double)(((int)st[7]) ^ parity);
    }
}

// Q[:, c0 .. c0+32) = H_0 ... H_{M-1} e_c, accumulated backwards in shared
// memory (reflector j only touches rows >= j and columns >= j).
__global__ void __launch_bounds__(256) k_form_q32(const float2* __restrict__ VT, const double* __restrict__ htau,
                                                 float* __restrict__ Ypl, float* __restrict__ Yf, int M, Planes P,
                                                 size_t wstride) {
    extern __shared__ unsigned char smem_raw[];
    float2* Qp = reinterpret_cast<float2*>(smem_raw);     // [M][QP]
    float2* ub = Qp + (size_t)M * QP;                     // [M]
    __shared__ float2 part[8][QP];
    __shared__ float2 wv[QP];
    const int tid = threadIdx.x;
    const int cc = tid & (QP - 1), g = tid >> 5;          // column in panel, row group (8 groups)
    const int w = blockIdx.y;
    const int c0 = blockIdx.x * QP;
    const int ncol = min(QP, M - c0);
    const long off = (long)w * M * M;
    const float2* V = VT + off;
    const double* tau = htau + (long)w * M;
    for (int e = tid; e < M * QP; e += blockDim.x) {
        const int r = e / QP, c = e % QP;
        Qp[e] = make_float2(r == c0 + c ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    const int jmax = c0 + ncol - 1;
    for (int j = jmax; j >= 0; --j) {
        for (int r = j + tid; r < M; r += blockDim.x) ub[r] = V[(long)j * M + r];
        __syncthreads();
        float2 s = make_float2(0.f, 0.f);
        if (cc < ncol && c0 + cc >= j)
            for (int r = j + g; r < M; r += 8) {
                const float2 u = ub[r], q = Qp[r * QP + cc];
                s.x = fmaf(u.x, q.x, fmaf(u.y, q.y, s.x));     // conj(u) q
                s.y = fmaf(u.x, q.y, fmaf(-u.y, q.x, s.y));
            }
        part[g][cc] = s;
        __syncthreads();
        if (g == 0) {
            float2 t = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 8; ++k) t = t + part[k][cc];
            const float tj = (float)tau[j];
            wv[cc] = make_float2(t.x * tj, t.y * tj);
        }
        __syncthreads();
        if (cc < ncol && c0 + cc >= j) {
            const float2 wc = wv[cc];
            for (int r = j + g; r < M; r += 8) {
                const float2 u = ub[r];
                float2 q = Qp[r * QP + cc];
                q.x = fmaf(-u.x, wc.x, fmaf(u.y, wc.y, q.x));
                q.y = fmaf(-u.x, wc.y, fmaf(-u.y, wc.x, q.y));
                Qp[r * QP + cc] = q;
            }
        }
        __syncthreads();
    }
    float* Yw = Ypl + wstride * w;
    for (int e = tid; e < ncol * M; e += blockDim.x) {
        const int c = e / M, i = e % M;
        const float2 q = Qp[i * QP + c];
        P.store(Yw, i, c0 + c, q);
        float* f = Yf + P.part * w + (size_t)(c0 + c) * (2 * P.Kp) + i;     // same value, one plane
        f[0] = q.x;
        f[P.Kp] = q.y;
    }
}

}  // namespace

cudaError_t launch_qr_prepiv(ftq_ctx* c) {
    const int M = c->M;
    Planes P;
    P.Kp = c->Kp;
    P.part = (size_t)c->LD * 2 * c->Kp;
    const size_t ws = 2 * P.part;
    int nt = (M + 31) / 32 * 32;
    nt = nt < 64 ? 64 : (nt > 288 ? 288 : nt);          // the launch bound; every loop strides by nt
    const size_t sm1 = (3 * NBJ + 1) * sizeof(double) * M + (sizeof(int) + 1) * M + 16;
    static size_t sm1_set = 48 * 1024;
    if (sm1 > sm1_set) {
        cudaError_t e = cudaFuncSetAttribute(k_qr_prepiv64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
        if (e != cudaSuccess) return e;
        sm1_set = sm1;
    }
    {
        LaunchScope ls(c, FTQ_K_QRCP);
        k_qr_prepiv64<<<c->W, nt, sm1, c->stream>>>(c->Ypl, c->work, c->work2, c->DR, c->Tinv, c->w2_32, c->htau,
                                                    c->xsum, c->wstate, c->status, M, P, ws);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t sm2 = sizeof(float2) * ((size_t)M * QP + M);
    static size_t sm2_set = 48 * 1024;
    if (sm2 > sm2_set) {
        e = cudaFuncSetAttribute(k_form_q32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        if (e != cudaSuccess) return e;
        sm2_set = sm2;
    }
    LaunchScope ls(c, FTQ_K_BRIDGE);
    k_form_q32<<<dim3((unsigned)((M + QP - 1) / QP), (unsigned)c->W), 256, sm2, c->stream>>>(c->w2_32, c->htau,
                                                                                          c->Ypl, c->Yf, M, P, ws);
    return cudaGetLastError();
}

}  // namespace ftq

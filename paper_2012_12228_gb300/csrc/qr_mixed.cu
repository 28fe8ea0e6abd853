// Stabilisation of the mixed-precision chain with pre-pivoting.
//
// The right block is A_R = Y D_R T with Y = (B's since the last QR) Q_R in
// FP32 and D_R, T^-1 in FP64.  Instead of pivoting at every Householder
// step, the columns of C = Y D_R are sorted once by their norms (the
// pre-pivoting of the GPU stratification work the paper cites for its
// stabilisation): C Pi has decreasing column norms, Y is well conditioned
// (a few B's times a unitary matrix) and the grading sits in D_R, so an
// unpivoted Householder QR of C Pi separates the scales like QRCP does.
// A column scaling only rescales R: with D' = Pi^T D_R Pi and
// Y Pi = Q R_Y, C Pi = Y Pi D' = Q (R_Y D').  So the reflectors and Q come
// from Y Pi alone, which is FP32-accurate, and are computed in FP32; the
// scales D_R = diag(R_Y) D', U = D^-1 R and the update of T^-1 stay in FP64.
//
//   k_prepiv32 (one block per walker): norms of C in FP64, ranks, parity,
//       D', and A = Y Pi (FP32, row-major).
//   k_qr32 (one block per walker): blocked Householder QR of A in FP32
//       (compact WY panels of NB columns); R_Y in A, reflectors and tau out.
//   k_tinv64 (FP64, one block per walker): D_R, U and T^-1 <- T^-1 Pi U^-1.
//   k_form_q32 (FP32, one block per walker and 32- or 16-column panel): Q = H_0 ...
//       H_{M-1} applied to the identity panel in shared memory, written into
//       the chain planes as the new Y.
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"
#include "mixed_common.cuh"

namespace ftq {
namespace {

constexpr int NBJ = 2;   // columns per block of the T^-1 update

// ---------------------------------------------------------------- S1: pre-pivoting
// Column norms of C = Y D_R (FP64 sums of the FP32 chain, a warp per column),
// the rank of every column (descending norm, ties to the lower index), the
// permutation's parity, D' = D_R Pi, and the permuted chain A = Y Pi written
// row-major in FP32 through 32 x 33 shared tiles (columns of Y are read
// contiguously, rows of A written contiguously).
__global__ void __launch_bounds__(256) k_prepiv32(const float* __restrict__ Ypl, float2* __restrict__ A,
                                                 const double2* __restrict__ DR, double2* __restrict__ Dp,
                                                 int* __restrict__ permg, double* __restrict__ ws,
                                                 int* __restrict__ status, int M, Planes P, size_t wstride,
                                                 int update_parity) {
    extern __shared__ unsigned char smem_raw[];
    double* cn = reinterpret_cast<double*>(smem_raw);                  // [M]
    float2* tile = reinterpret_cast<float2*>(cn + M);                 // [32][33]
    int* perm = reinterpret_cast<int*>(tile + 32 * 33);               // [M]
    unsigned char* seen = reinterpret_cast<unsigned char*>(perm + M);   // [M]
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int w = blockIdx.x;
    const float* Yw = Ypl + wstride * w;
    const double2* Dw = DR + (long)w * M;
    for (int c = warp; c < M; c += nw) {
        double sum = 0.0;
        for (int i = lane; i < M; i += 32) {
            const float2 y = P.load(Yw, i, c);
            sum += (double)y.x * y.x + (double)y.y * y.y;
        }
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            double v = sum * abs2(Dw[c]);
            // a NaN norm would compare false both ways and give two columns one
            // rank (leaving an entry of perm unset); rank it last and latch
            if (v != v) {
                v = -INFINITY;
                atomicOr(status, 1);
            }
            cn[c] = v;
        }
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
    if (tid == 0 && update_parity) {
        // parity of the permutation = (M - number of cycles) mod 2
        int cycles = 0;
        for (int c = 0; c < M; ++c) {
            if (seen[c]) continue;
            ++cycles;
            for (int x = c; !seen[x]; x = perm[x]) seen[x] = 1;
        }
        double* st = ws + (long)WSTRIDE * w;
        st[7] = (double)(((int)st[7]) ^ ((M - cycles) & 1));
    }
    for (int j = tid; j < M; j += nt) {
        permg[(long)w * M + j] = perm[j];
        Dp[(long)w * M + j] = Dw[perm[j]];
    }
    float2* Aw = A + (long)w * M * M;
    const int nt32 = (M + 31) / 32;
    for (int t = 0; t < nt32 * nt32; ++t) {
        const int i0 = (t / nt32) * 32, j0 = (t % nt32) * 32;
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += nt) {
            const int jj = e >> 5, ii = e & 31;                // read column perm[j0 + jj], rows i0 + ii
            const int i = i0 + ii, j = j0 + jj;
            tile[jj * 33 + ii] = (i < M && j < M) ? P.load(Yw, i, perm[j]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += nt) {
            const int ii = e >> 5, jj = e & 31;                // write row i0 + ii, columns j0 + jj
            const int i = i0 + ii, j = j0 + jj;
            if (i < M && j < M) Aw[(long)i * M + j] = tile[jj * 33 + ii];
        }
    }
}

// ---------------------------------------------------------------- S2: FP32 blocked Householder QR
// Householder QR of A = Y Pi (M x M, row-major, FP32), one block per walker,
// NB-column panels.  A panel (rows j0.., NB columns) is factorised in shared
// memory (a reflector per column: beta = -|x| x_0/|x_0| replaces the
// diagonal, u = x - beta e_0, tau = 1/(|x| (|x| + |x_0|)), H = I - tau u u^H
// Hermitian); T of the compact form H_0 ... H_{nb-1} = I - V T V^H is built
// from the Gram matrix of V; the trailing columns then take all nb
// reflectors at once, A <- A - V T^H (V^H A), one column per thread, V read
// from shared memory (the same row for every thread: a broadcast), so each
// column is read twice and written once per panel.  Outputs: R in the upper
// triangle of A, the reflectors as rows VT[j][r] (r >= j, u_0 at r = j) and
// tau in FP64 for the Q panels.
template <int NB>
__global__ void __launch_bounds__(256, 1) k_qr32(float2* __restrict__ A, float2* __restrict__ VT,
                                                double* __restrict__ htau, int* __restrict__ status, int M) {
    extern __shared__ unsigned char smem_raw[];
    float2* V = reinterpret_cast<float2*>(smem_raw);        // [M][NB]  panel, then the reflectors
    float2* Yt = V + (size_t)M * NB;                        // [M][NB]  V T^H
    __shared__ float2 T[NB][NB + 1];
    __shared__ float2 Sg[NB][NB + 1];
    __shared__ float tau_s[NB];
    __shared__ float2 beta_s[NB];
    __shared__ float red[32];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int w = blockIdx.x;
    float2* Aw = A + (long)w * M * M;
    float2* Vw = VT + (long)w * M * M;
    double* tw = htau + (long)w * M;
    for (int e = tid; e < NB * (NB + 1); e += nt) (&T[0][0])[e] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < M; j0 += NB) {
        const int nb = min(NB, M - j0), rows = M - j0;
        for (int e = tid; e < rows * NB; e += nt) {
            const int r = e / NB, c = e % NB;
            V[e] = c < nb ? Aw[(long)(j0 + r) * M + j0 + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // unblocked factorisation of the panel
        for (int c = 0; c < nb; ++c) {
            float s = 0.f;
            for (int r = c + tid; r < rows; r += nt) {
                const float2 x = V[r * NB + c];
                s = fmaf(x.x, x.x, fmaf(x.y, x.y, s));
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp] = s;
            __syncthreads();
            if (tid == 0) {
                float tot = 0.f;
                for (int q = 0; q < nw; ++q) tot += red[q];
                const float2 al = V[c * NB + c];
                const float sig = sqrtf(tot);
                const float aa = sqrtf(al.x * al.x + al.y * al.y);
                const float2 be = aa > 0.f ? make_float2(-sig * al.x / aa, -sig * al.y / aa) : make_float2(-sig, 0.f);
                const float uhu = sig * (sig + aa);
                tau_s[c] = uhu > 0.f ? 1.f / uhu : 0.f;
                beta_s[c] = be;
                V[c * NB + c] = make_float2(al.x - be.x, al.y - be.y);     // u_0
                if (!(sig > 0.f)) atomicOr(status, 1);
            }
            __syncthreads();
            const float tc = tau_s[c];
            for (int c2 = c + 1 + warp; c2 < nb; c2 += nw) {
                float dx = 0.f, dy = 0.f;                              // u^H x
                for (int r = c + lane; r < rows; r += 32) {
                    const float2 u = V[r * NB + c], x = V[r * NB + c2];
                    dx = fmaf(u.x, x.x, fmaf(u.y, x.y, dx));
                    dy = fmaf(u.x, x.y, fmaf(-u.y, x.x, dy));
                }
                for (int o = 16; o > 0; o >>= 1) {
                    dx += __shfl_xor_sync(0xffffffffu, dx, o);
                    dy += __shfl_xor_sync(0xffffffffu, dy, o);
                }
                dx *= tc;
                dy *= tc;
                for (int r = c + lane; r < rows; r += 32) {
                    const float2 u = V[r * NB + c];
                    float2 x = V[r * NB + c2];
                    x.x = fmaf(-u.x, dx, fmaf(u.y, dy, x.x));
                    x.y = fmaf(-u.x, dy, fmaf(-u.y, dx, x.y));
                    V[r * NB + c2] = x;
                }
            }
            __syncthreads();
        }
        // R rows of the panel and the reflectors out; V keeps only the reflectors
        for (int e = tid; e < rows * NB; e += nt) {
            const int r = e / NB, c = e % NB;
            if (c >= nb) continue;
            const float2 v = V[e];
            if (r < c) {
                Aw[(long)(j0 + r) * M + j0 + c] = v;                     // R above the diagonal
                V[e] = make_float2(0.f, 0.f);
            } else {
                Vw[(long)(j0 + c) * M + j0 + r] = v;
                if (r == c) Aw[(long)(j0 + r) * M + j0 + c] = beta_s[c];
            }
        }
        for (int c = tid; c < nb; c += nt) tw[j0 + c] = (double)tau_s[c];
        __syncthreads();
        if (j0 + nb >= M) break;
        // Gram matrix S = V^H V (upper part) and T: T_cc = tau_c,
        // T[0:c, c] = -tau_c T[0:c, 0:c] S[0:c, c]
        for (int q = warp; q < nb * nb; q += nw) {
            const int a = q / nb, b = q % nb;
            if (a >= b) continue;
            float sx = 0.f, sy = 0.f;
            for (int r = b + lane; r < rows; r += 32) {
                const float2 u = V[r * NB + a], x = V[r * NB + b];
                sx = fmaf(u.x, x.x, fmaf(u.y, x.y, sx));
                sy = fmaf(u.x, x.y, fmaf(-u.y, x.x, sy));
            }
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0) Sg[a][b] = make_float2(sx, sy);
        }
        __syncthreads();
        if (warp == 0) {
            for (int c = 0; c < nb; ++c) {
                // lane a < c: T[a][c] = -tau_c sum_{b = a .. c-1} T[a][b] S[b][c]
                float2 t = make_float2(0.f, 0.f);
                if (lane < c) {
                    for (int b = lane; b < c; ++b) {
                        const float2 x = T[lane][b], y = Sg[b][c];
                        t.x = fmaf(x.x, y.x, fmaf(-x.y, y.y, t.x));
                        t.y = fmaf(x.x, y.y, fmaf(x.y, y.x, t.y));
                    }
                }
                __syncwarp();
                if (lane < c) T[lane][c] = make_float2(-tau_s[c] * t.x, -tau_s[c] * t.y);
                if (lane == c) T[c][c] = make_float2(tau_s[c], 0.f);
                if (lane > c && lane < NB) T[lane][c] = make_float2(0.f, 0.f);
                __syncwarp();
            }
        }
        __syncthreads();
        // Yt = V T^H: Yt[r][c] = sum_{b >= c} V[r][b] conj(T[c][b])
        for (int e = tid; e < rows * NB; e += nt) {
            const int r = e / NB, c = e % NB;
            float2 t = make_float2(0.f, 0.f);
            for (int b = c; b < NB; ++b) {
                const float2 v = V[r * NB + b], x = T[c][b];
                t.x = fmaf(v.x, x.x, fmaf(v.y, x.y, t.x));
                t.y = fmaf(v.y, x.x, fmaf(-v.x, x.y, t.y));
            }
            Yt[e] = t;
        }
        __syncthreads();
        // trailing columns: w = V^H a, then a <- a - (V T^H) w
        for (int col = j0 + nb + tid; col < M; col += nt) {
            float2 wv[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) wv[c] = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int r = 0; r < rows; ++r) {
                const float2 a = Aw[(long)(j0 + r) * M + col];
                const float2* vr = V + r * NB;
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const float2 u = vr[c];                            // conj(u) a
                    wv[c].x = fmaf(u.x, a.x, fmaf(u.y, a.y, wv[c].x));
                    wv[c].y = fmaf(u.x, a.y, fmaf(-u.y, a.x, wv[c].y));
                }
            }
#pragma unroll 1
            for (int r = 0; r < rows; ++r) {
                float2 a = Aw[(long)(j0 + r) * M + col];
                const float2* yr = Yt + r * NB;
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const float2 u = yr[c];
                    a.x = fmaf(-u.x, wv[c].x, fmaf(u.y, wv[c].y, a.x));
                    a.y = fmaf(-u.x, wv[c].y, fmaf(-u.y, wv[c].x, a.y));
                }
                Aw[(long)(j0 + r) * M + col] = a;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- S3: FP64 update of the right block
// From R_Y (upper triangle of A, FP32) and D' (FP64): D_R <- diag(R_Y) D',
// U = D^-1 R with R = R_Y D', i.e. U_mj = (R_Y[m][j] / R_Y[m][m]) (D'_j / D'_m)
// in FP64, and T^-1 <- T^-1 Pi U^-1 by the blocked column solve below.
__global__ void __launch_bounds__(288, 4) k_tinv64(const float2* __restrict__ A, const double2* __restrict__ Dp,
                                                  const int* __restrict__ permg, double2* __restrict__ work,
                                                  double2* __restrict__ work2, double2* __restrict__ DR,
                                                  double2* __restrict__ Tinv, double* __restrict__ xsum,
                                                  int* __restrict__ status, int M) {
    extern __shared__ unsigned char smem_raw[];
    double* ub = reinterpret_cast<double*>(smem_raw);      // [M][NBJ][3] U block of the T^-1 update
    double2* dinv = reinterpret_cast<double2*>(ub + 3 * NBJ * M);   // [M] 1 / (R_Y[m][m] D'_m)
    int* perm = reinterpret_cast<int*>(dinv + M);          // [M]
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w = blockIdx.x;
    const long off = (long)w * M * M;
    const float2* Aw = A + off;
    double2* C = work + off;
    double2* XT = work2 + off;
    double2* Ti = Tinv + off;
    const double2* Dpw = Dp + (long)w * M;
    for (int j = tid; j < M; j += nt) {
        const float2 r = Aw[(long)j * M + j];
        const double2 d = cmul(make_double2(r.x, r.y), Dpw[j]);
        DR[(long)w * M + j] = d;
        if (!(abs2(d) > 0.0)) atomicOr(status, 1);
        dinv[j] = cinv(d);
        perm[j] = permg[(long)w * M + j];
    }
    __syncthreads();
    // U in the strict upper triangle of C, Re U + Im U in the real parts of
    // the lower triangle: U[m][j] -> C[j][m].x
    for (long e = tid; e < (long)M * M; e += nt) {
        const int m = (int)(e / M), j = (int)(e % M);
        if (j > m) {
            const float2 r = Aw[e];
            const double2 u = cmul(cmul(make_double2(r.x, r.y), Dpw[j]), dinv[m]);
            C[e] = u;
            C[(long)j * M + m].x = u.x + u.y;
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
}

// ---------------------------------------------------------------- S3 in double-FP32
// The same update, T^-1 <- T^-1 Pi U^-1 (X U = Z, Z = T^-1 Pi), with every
// value carried as an unevaluated sum of two floats (hi + lo, 48 significand
// bits) on the FP32 pipe, whose rate on this part is 64 times that of the
// FP64 pipe.  Products are split exactly with FMA (Dekker / Knuth two-product,
// two-sum; the lo * lo term, 2^-48 relative, is dropped) and the running sums
// carry their rounding errors in the lo part.
//
// k_udt_prep (one block per walker): D_R = diag(R_Y) D', U_mj =
//   (R_Y[m][j] / R_Y[m][m]) (D'_j / D'_m) formed in FP64 and stored as
//   double-FP32 (Re hi, Re lo, Im hi, Im lo) in the upper triangle.
// k_tinv_df (a block per walker and row range, one row of X per thread): the
//   forward solve in NBJ-column blocks, the block's strip of U staged in
//   shared memory and read at the same address by every thread; X column-major
//   in double-FP32 in the scratch; T^-1 rows written back in FP64 through a
//   shared tile.
struct df2 { float h, l; };

__device__ __forceinline__ df2 df_split(double v) {
    df2 r;
    r.h = (float)v;
    r.l = (float)(v - (double)r.h);
    return r;
}

// acc -= x * u  (x, u double-FP32; acc.l collects the rounding errors)
__device__ __forceinline__ void df_msub(df2& acc, float xh, float xl, float uh, float ul) {
    const float p = xh * uh;
    float e = fmaf(xh, uh, -p);
    e = fmaf(xh, ul, e);
    e = fmaf(xl, uh, e);
    const float t = acc.h - p;
    const float bb = t - acc.h;
    const float err = (acc.h - (t - bb)) + (-p - bb);
    acc.h = t;
    acc.l += err - e;
}

// acc += x * u
__device__ __forceinline__ void df_madd(df2& acc, float xh, float xl, float uh, float ul) {
    df_msub(acc, -xh, -xl, uh, ul);
}

__device__ __forceinline__ df2 df_norm(df2 a) {
    df2 r;
    r.h = a.h + a.l;
    r.l = a.l - (r.h - a.h);
    return r;
}

__global__ void __launch_bounds__(256) k_udt_prep(const float2* __restrict__ A, const double2* __restrict__ Dp,
                                                 float4* __restrict__ Udf, double2* __restrict__ DR,
                                                 int* __restrict__ status, int M) {
    extern __shared__ unsigned char smem_raw[];
    double2* dinv = reinterpret_cast<double2*>(smem_raw);   // [M] 1 / (R_Y[m][m] D'_m)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w = blockIdx.x;
    const long off = (long)w * M * M;
    const float2* Aw = A + off;
    const double2* Dpw = Dp + (long)w * M;
    for (int j = tid; j < M; j += nt) {
        const float2 r = Aw[(long)j * M + j];
        const double2 d = cmul(make_double2(r.x, r.y), Dpw[j]);
        DR[(long)w * M + j] = d;
        if (!(abs2(d) > 0.0)) atomicOr(status, 1);
        dinv[j] = cinv(d);
    }
    __syncthreads();
    float4* U = Udf + off;
    for (long e = tid; e < (long)M * M; e += nt) {
        const int m = (int)(e / M), j = (int)(e % M);
        if (j > m) {
            const float2 r = Aw[e];
            const double2 u = cmul(cmul(make_double2(r.x, r.y), Dpw[j]), dinv[m]);
            const df2 re = df_split(u.x), im = df_split(u.y);
            U[e] = make_float4(re.h, re.l, im.h, im.l);
        }
    }
}

template <int NBJ>
__global__ void __launch_bounds__(128) k_tinv_df(const float4* __restrict__ Udf, const int* __restrict__ permg,
                                                 float4* __restrict__ Xs, double2* __restrict__ Tinv,
                                                 int* __restrict__ status, int M) {
    extern __shared__ unsigned char smem_raw[];
    const int RB = blockDim.x;
    // the strip of U ([M][NBJ] float4) and, at the end, the output tile
    // ([16][RB + 1] double2, 16 bytes each as well) share the first region
    const size_t sreg = max((size_t)M * NBJ, (size_t)16 * (RB + 1));
    float4* S = reinterpret_cast<float4*>(smem_raw);
    int* perm = reinterpret_cast<int*>(S + sreg);           // [M]
    const int tid = threadIdx.x, w = blockIdx.y;
    const int i = blockIdx.x * RB + tid;
    const bool row = i < M;
    const long off = (long)w * M * M;
    const float4* U = Udf + off;
    float4* X = Xs + off;
    double2* Ti = Tinv + off;
    for (int m = tid; m < M; m += RB) perm[m] = permg[(long)w * M + m];
    bool bad = false;
    for (int jb = 0; jb < M; jb += NBJ) {
        const int nb = min(NBJ, M - jb);
        __syncthreads();
        for (int e = tid; e < (jb + nb) * NBJ; e += RB) {   // columns q >= nb and the lower part zero
            const int m = e / NBJ, q = e % NBJ;
            S[e] = (q < nb && m < jb + q) ? U[(long)m * M + jb + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        if (!row) continue;
        df2 sr[NBJ], si[NBJ];
#pragma unroll
        for (int q = 0; q < NBJ; ++q) {
            const double2 z = q < nb ? Ti[(long)i * M + perm[jb + q]] : make_double2(0.0, 0.0);
            sr[q] = df_split(z.x);
            si[q] = df_split(z.y);
        }
        for (int m = 0; m < jb; ++m) {
            const float4 x = X[(long)m * M + i];
            const float4* ur = S + m * NBJ;
#pragma unroll
            for (int q = 0; q < NBJ; ++q) {
                const float4 u = ur[q];
                // s -= x u: Re -= xr ur - xi ui, Im -= xr ui + xi ur
                df_msub(sr[q], x.x, x.y, u.x, u.y);
                df_madd(sr[q], x.z, x.w, u.z, u.w);
                df_msub(si[q], x.x, x.y, u.z, u.w);
                df_msub(si[q], x.z, x.w, u.x, u.y);
            }
        }
#pragma unroll
        for (int q = 0; q < NBJ; ++q) {
            if (q >= nb) continue;
#pragma unroll
            for (int q2 = 0; q2 < NBJ; ++q2) {
                if (q2 >= q) continue;
                const float4 u = S[(jb + q2) * NBJ + q];
                const df2 xr = sr[q2], xi = si[q2];
                df_msub(sr[q], xr.h, xr.l, u.x, u.y);
                df_madd(sr[q], xi.h, xi.l, u.z, u.w);
                df_msub(si[q], xr.h, xr.l, u.z, u.w);
                df_msub(si[q], xi.h, xi.l, u.x, u.y);
            }
            sr[q] = df_norm(sr[q]);
            si[q] = df_norm(si[q]);
        }
#pragma unroll
        for (int q = 0; q < NBJ; ++q)
            if (q < nb) {
                X[(long)(jb + q) * M + i] = make_float4(sr[q].h, sr[q].l, si[q].h, si[q].l);
                bad = bad || !isfinite(sr[q].h) || !isfinite(si[q].h);
            }
    }
    if (bad) atomicOr(status, 1);
    // T^-1 rows of this block in FP64 (hi + lo), 16 columns at a time through the tile
    double2* tile = reinterpret_cast<double2*>(S);
    const int r0 = blockIdx.x * RB;
    const int nrow = min(RB, M - r0);
    for (int cb = 0; cb < M; cb += 16) {
        __syncthreads();
        if (row)
            for (int cc = 0; cc < 16; ++cc)
                if (cb + cc < M) {
                    const float4 x = X[(long)(cb + cc) * M + i];
                    tile[cc * (RB + 1) + tid] = make_double2((double)x.x + (double)x.y, (double)x.z + (double)x.w);
                }
        __syncthreads();
        for (int e = tid; e < nrow * 16; e += RB) {
            const int r = e >> 4, cc = e & 15;
            if (cb + cc < M) Ti[(long)(r0 + r) * M + cb + cc] = tile[cc * (RB + 1) + r];
        }
    }
}

// Q[:, c0 .. c0+QP) = H_0 ... H_{M-1} e_c, accumulated backwards in shared
// memory (reflector j only touches rows >= j and columns >= j); 256 threads
// as QP columns x (256 / QP) row groups.
template <int QP>
__global__ void __launch_bounds__(256) k_form_q32(const float2* __restrict__ VT, const double* __restrict__ htau,
                                                 float* __restrict__ Ypl, float* __restrict__ Yf, int M, Planes P,
                                                 size_t wstride) {
    extern __shared__ unsigned char smem_raw[];
    float2* Qp = reinterpret_cast<float2*>(smem_raw);     // [M][QP]
    float2* ub = Qp + (size_t)M * QP;                     // [M]
    constexpr int NG = 256 / QP;                          // row groups
    __shared__ float2 part[NG][QP];
    __shared__ float2 wv[QP];
    const int tid = threadIdx.x;
    const int cc = tid & (QP - 1), g = tid / QP;          // column in panel, row group
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
            for (int r = j + g; r < M; r += NG) {
                const float2 u = ub[r], q = Qp[r * QP + cc];
                s.x = fmaf(u.x, q.x, fmaf(u.y, q.y, s.x));     // conj(u) q
                s.y = fmaf(u.x, q.y, fmaf(-u.y, q.x, s.y));
            }
        part[g][cc] = s;
        __syncthreads();
        if (g == 0) {
            float2 t = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NG; ++k) t = t + part[k][cc];
            const float tj = (float)tau[j];
            wv[cc] = make_float2(t.x * tj, t.y * tj);
        }
        __syncthreads();
        if (cc < ncol && c0 + cc >= j) {
            const float2 wc = wv[cc];
            for (int r = j + g; r < M; r += NG) {
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

bool qr_width_fits(int M, int nb) { return 2 * sizeof(float2) * (size_t)M * nb <= 200 * 1024; }

// The context's panel width when it fits (autotuned), else the widest that fits.
int qr_panel_width(const ftq_ctx* c) {
    if (c->qr_nb > 0 && qr_width_fits(c->M, c->qr_nb)) return c->qr_nb;
    for (int nb = 32; nb > 8; nb >>= 1)
        if (qr_width_fits(c->M, nb)) return nb;
    return 8;
}

cudaError_t launch_qr32(ftq_ctx* c, int nbq) {
    const int M = c->M;
    const size_t smq = 2 * sizeof(float2) * (size_t)M * nbq;
    static size_t smq_set[3] = {48 * 1024, 48 * 1024, 48 * 1024};
    const int which = nbq == 32 ? 0 : (nbq == 16 ? 1 : 2);
    cudaError_t e;
    if (smq > smq_set[which]) {
        e = nbq == 32 ? cudaFuncSetAttribute(k_qr32<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq)
            : nbq == 16 ? cudaFuncSetAttribute(k_qr32<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq)
                        : cudaFuncSetAttribute(k_qr32<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq);
        if (e != cudaSuccess) return e;
        smq_set[which] = smq;
    }
    if (nbq == 32) k_qr32<32><<<c->W, 256, smq, c->stream>>>(c->w32, c->w2_32, c->htau, c->status, M);
    else if (nbq == 16) k_qr32<16><<<c->W, 256, smq, c->stream>>>(c->w32, c->w2_32, c->htau, c->status, M);
    else k_qr32<8><<<c->W, 256, smq, c->stream>>>(c->w32, c->w2_32, c->htau, c->status, M);
    return cudaGetLastError();
}

cudaError_t launch_prepiv(ftq_ctx* c, bool update_parity = true) {
    const int M = c->M;
    Planes P;
    P.Kp = c->Kp;
    P.part = (size_t)c->LD * 2 * c->Kp;
    const size_t sm0 = (sizeof(double) + sizeof(int) + 1) * M + sizeof(float2) * 32 * 33 + 16;
    static size_t sm0_set = 48 * 1024;
    if (sm0 > sm0_set) {
        cudaError_t e = cudaFuncSetAttribute(k_prepiv32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0);
        if (e != cudaSuccess) return e;
        sm0_set = sm0;
    }
    k_prepiv32<<<c->W, 256, sm0, c->stream>>>(c->Ypl, c->w32, c->DR, c->hh, c->perm, c->wstate, c->status, M, P,
                                              2 * P.part, update_parity ? 1 : 0);
    return cudaGetLastError();
}

// Time the FP32 QR for every panel width that fits (on the walkers' current
// chain, re-pivoted before each trial; the T^-1 update is not run, so the
// state is unchanged) and keep the fastest.
cudaError_t qr_autotune(ftq_ctx* c, int* best_nb, float* best_ms) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaSuccess;
    int best = 0;
    float bms = 1e30f;
    for (int nb = 32; nb >= 8; nb >>= 1) {
        if (!qr_width_fits(c->M, nb)) continue;
        e = launch_prepiv(c, false);
        if (e == cudaSuccess) e = launch_qr32(c, nb);     // warm-up
        if (e == cudaSuccess) e = launch_prepiv(c, false);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = launch_qr32(c, nb);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < bms) { bms = ms; best = nb; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    c->qr_nb = best;
    *best_nb = best;
    *best_ms = bms;
    return cudaSuccess;
}

constexpr int TNBJ = 8;   // columns per block of the double-FP32 solve

size_t tinv_df_smem(int M, int RB) {
    const size_t sreg = (size_t)M * TNBJ > (size_t)16 * (RB + 1) ? (size_t)M * TNBJ : (size_t)16 * (RB + 1);
    return sizeof(float4) * sreg + sizeof(int) * M;
}

cudaError_t launch_tinv_df(ftq_ctx* c) {
    const int M = c->M;
    float4* U = reinterpret_cast<float4*>(c->work);       // double-FP32 U, [W][M][M] (16 bytes per entry)
    float4* X = reinterpret_cast<float4*>(c->work2);      // double-FP32 X, column-major
    const size_t sm0 = sizeof(double2) * M;
    static size_t sm0_set = 48 * 1024;
    cudaError_t e;
    if (sm0 > sm0_set) {
        e = cudaFuncSetAttribute(k_udt_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0);
        if (e != cudaSuccess) return e;
        sm0_set = sm0;
    }
    k_udt_prep<<<c->W, 256, sm0, c->stream>>>(c->w32, c->hh, U, c->DR, c->status, M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nblk = (M + 127) / 128;
    const int RB = ((M + nblk - 1) / nblk + 31) / 32 * 32;     // rows per block, <= 128
    const size_t sm = tinv_df_smem(M, RB);
    static size_t sm_set = 48 * 1024;
    if (sm > sm_set) {
        e = cudaFuncSetAttribute(k_tinv_df<TNBJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        sm_set = sm;
    }
    k_tinv_df<TNBJ><<<dim3((unsigned)nblk, (unsigned)c->W), RB, sm, c->stream>>>(U, c->perm, X, c->Tinv, c->status, M);
    return cudaGetLastError();
}

cudaError_t launch_qr_prepiv(ftq_ctx* c) {
    const int M = c->M;
    Planes P;
    P.Kp = c->Kp;
    P.part = (size_t)c->LD * 2 * c->Kp;
    const size_t ws = 2 * P.part;
    cudaError_t e;
    {
        LaunchScope ls(c, FTQ_K_QRCP);
        e = launch_prepiv(c);
        if (e != cudaSuccess) return e;
        e = launch_qr32(c, qr_panel_width(c));
        if (e != cudaSuccess) return e;
    }
    if (c->opts.precision != FTQ_MIXED_F64UDT) {
        LaunchScope ls(c, FTQ_K_TINV);
        e = launch_tinv_df(c);
        if (e != cudaSuccess) return e;
    } else {
        LaunchScope ls(c, FTQ_K_TINV);
        int nt = (M + 31) / 32 * 32;
        nt = nt < 64 ? 64 : (nt > 288 ? 288 : nt);          // the launch bound; every loop strides by nt
        const size_t sm1 = 3 * NBJ * sizeof(double) * M + sizeof(double2) * M + sizeof(int) * M + 16;
        static size_t sm1_set = 48 * 1024;
        if (sm1 > sm1_set) {
            e = cudaFuncSetAttribute(k_tinv64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
            if (e != cudaSuccess) return e;
            sm1_set = sm1;
        }
        k_tinv64<<<c->W, nt, sm1, c->stream>>>(c->w32, c->hh, c->perm, c->work, c->work2, c->DR, c->Tinv, c->xsum,
                                               c->status, M);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // 32-column Q panels while they fit in shared memory, else 16
    const bool wide = sizeof(float2) * ((size_t)M * 32 + M) <= 200 * 1024;
    const int QP = wide ? 32 : 16;
    const size_t sm2 = sizeof(float2) * ((size_t)M * QP + M);
    static size_t sm2_set[2] = {48 * 1024, 48 * 1024};
    if (sm2 > sm2_set[wide]) {
        e = wide ? cudaFuncSetAttribute(k_form_q32<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)
                 : cudaFuncSetAttribute(k_form_q32<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        if (e != cudaSuccess) return e;
        sm2_set[wide] = sm2;
    }
    LaunchScope ls(c, FTQ_K_BRIDGE);
    const dim3 grid((unsigned)((M + QP - 1) / QP), (unsigned)c->W);
    if (wide) k_form_q32<32><<<grid, 256, sm2, c->stream>>>(c->w2_32, c->htau, c->Ypl, c->Yf, M, P, ws);
    else k_form_q32<16><<<grid, 256, sm2, c->stream>>>(c->w2_32, c->htau, c->Ypl, c->Yf, M, P, ws);
    return cudaGetLastError();
}

}  // namespace ftq

// Low-rank truncation of the complex128 path (Sec. "Exploiting the low-rank
// structure", Eq. thresh, with the Woodbury identity and the matrix
// determinant lemma).
//
// The right block is R = Y diag(D) T with Y M x m, D m and T m x M (T itself,
// rows 0..m-1 of the buffer that holds T^-1 on the full-rank path); m is the
// walker's rank, kept in its state record.  Every stabilisation QR-factorises
// the M x m panel Y D with column pivoting and keeps the leading columns with
// |R_jj| >= threshold (at least one).  The left block D_L = B_T^p keeps its
// entries >= threshold (m_L of them, index list L).  Then, in the cyclic
// order G(tau) = (I + R D_L)^-1:
//   core c = D T[:, L] d_L (m x m_L), QRCP c = q_c r_c pi_c (m_T = min(m, m_L)),
//   q = Y q_c (M x m_T), d = diag r_c, t = (d^-1 r_c)(pi_c P_L^T) (m_T x M),
//   X = t q, I + d X = d_b^-1 (d_b + d_s X) with the split of the stable G,
//   G = I - q (d_b + d_s X)^-1 d_s t,
//   ln det(I + A) = ln det(d_b + d_s X) - sum ln d_b.
// One thread block per walker, as the full-rank factorisations.
#include <cmath>
#include <vector>

#include "block_reduce.cuh"
#include "complex_math.cuh"
#include "ftq_internal.h"

namespace ftq {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Householder step on column j of the row-major panel A (leading dimension
// ld), rows j..rows-1: H = I - tau u u^H with u = x - beta e_1,
// beta = -e^{i arg x_0} |x|; stores u_0 in u0[j], tau[j], A[j][j] = beta and
// leaves u's tail in A[j+1.., j].  sq = |x|^2 (the pivot column's norm).
__device__ void reflector(double2* A, int ld, int j, double sq, double2* u0, double* tau, int* status) {
    const double2 al = A[(long)j * ld + j];
    const double sig = sqrt(sq);
    const double aa = sqrt(abs2(al));
    const double2 beta = aa > 0.0 ? al * (-sig / aa) : make_double2(-sig, 0.0);
    const double uhu = 2.0 * sig * (sig + aa);
    u0[j] = al - beta;
    tau[j] = uhu > 0.0 ? 2.0 / uhu : 0.0;
    A[(long)j * ld + j] = beta;
    if (!(sig > 0.0)) atomicOr(status, 1);
}

// Businger-Golub QRCP of the rows x cols panel A (row-major, leading
// dimension ld) for kmax = min(rows, cols) steps: pivot = remaining column of
// largest norm, ties to the lowest index; perm[j] = original column of
// position j.  Returns the row-swap-free parity of the column permutation.
__device__ int qrcp_panel(double2* A, int ld, int rows, int cols, int kmax, int* perm, double* cn, double2* u0,
                          double* tau, double* shv, int* shi, int* status) {
    const int nt = blockDim.x;
    __shared__ int nswap;
    for (int c = threadIdx.x; c < cols; c += nt) perm[c] = c;
    if (threadIdx.x == 0) nswap = 0;
    __syncthreads();
    for (int j = 0; j < kmax; ++j) {
        double best = -1.0;
        int bidx = cols;
        for (int c = j + threadIdx.x; c < cols; c += nt) {
            double s = 0.0;
            for (int r = j; r < rows; ++r) s += abs2(A[(long)r * ld + c]);
            cn[c] = s;
            if (s > best) { best = s; bidx = c; }
        }
        int pc = block_argmax(best, bidx, shv, shi);
        if (pc >= cols) {                    // every candidate norm was NaN
            pc = j;
            if (threadIdx.x == 0) atomicOr(status, 1);
        }
        if (pc != j) {
            for (int r = threadIdx.x; r < rows; r += nt) {
                double2 t = A[(long)r * ld + j];
                A[(long)r * ld + j] = A[(long)r * ld + pc];
                A[(long)r * ld + pc] = t;
            }
            if (threadIdx.x == 0) {
                int t = perm[j]; perm[j] = perm[pc]; perm[pc] = t;
                double tn = cn[j]; cn[j] = cn[pc]; cn[pc] = tn;
                nswap ^= 1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) reflector(A, ld, j, cn[j], u0, tau, status);
        __syncthreads();
        const double2 uj = u0[j];
        const double tj = tau[j];
        for (int c = j + 1 + threadIdx.x; c < cols; c += nt) {
            double2 s = cmul(conj(uj), A[(long)j * ld + c]);
            for (int r = j + 1; r < rows; ++r) s = cfma(conj(A[(long)r * ld + j]), A[(long)r * ld + c], s);
            s = s * tj;
            A[(long)j * ld + c] = cfms(uj, s, A[(long)j * ld + c]);
            for (int r = j + 1; r < rows; ++r) A[(long)r * ld + c] = cfms(A[(long)r * ld + j], s, A[(long)r * ld + c]);
        }
        __syncthreads();
    }
    const int par = nswap;
    __syncthreads();
    return par;
}

// Q (rows x kmax, leading dimension ld) = H_0 ... H_{kmax-1} applied to the
// first kmax columns of the identity (backward accumulation); the reflector
// tails sit below the diagonal of A.
__device__ void form_q(const double2* A, int lda, double2* Q, int ldq, int rows, int kmax, const double2* u0,
                       const double* tau) {
    const int nt = blockDim.x;
    for (long e = threadIdx.x; e < (long)rows * kmax; e += nt) {
        int i = (int)(e / kmax), c = (int)(e % kmax);
        Q[(long)i * ldq + c] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int j = kmax - 1; j >= 0; --j) {
        const double2 uj = u0[j];
        const double tj = tau[j];
        for (int c = j + threadIdx.x; c < kmax; c += nt) {
            double2 s = cmul(conj(uj), Q[(long)j * ldq + c]);
            for (int r = j + 1; r < rows; ++r) s = cfma(conj(A[(long)r * lda + j]), Q[(long)r * ldq + c], s);
            s = s * tj;
            Q[(long)j * ldq + c] = cfms(uj, s, Q[(long)j * ldq + c]);
            for (int r = j + 1; r < rows; ++r) Q[(long)r * ldq + c] = cfms(A[(long)r * lda + j], s, Q[(long)r * ldq + c]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- stabilisation
// QRCP of C = Y[:, :m] diag(D) (M x m); D <- diag R over the kept prefix
// |R_jj| >= thr (at least one), T <- (D^-1 R)(Pi T) restricted to the kept
// rows, Q -> Qout (first m' columns), rank m' -> ws[12].
constexpr int LR_THREADS = 512;

__global__ void __launch_bounds__(LR_THREADS) k_qrcp_lr(const double2* __restrict__ Yin, double2* __restrict__ Qout, double2* __restrict__ work,
                          double2* __restrict__ work2, double2* __restrict__ DR, double2* __restrict__ Tm,
                          double2* __restrict__ hh, double* __restrict__ htau, double* __restrict__ ws,
                          int* __restrict__ status, int M, double thr) {
    extern __shared__ unsigned char smem_raw[];
    double* cn = reinterpret_cast<double*>(smem_raw);          // [M]
    int* perm = reinterpret_cast<int*>(cn + M);                 // [M]
    __shared__ double shv[32];
    __shared__ int shi[32];
    __shared__ int mnew;
    const int w = blockIdx.x, nt = blockDim.x;
    const long off = (long)w * M * M;
    double* s = ws + (long)WSTRIDE * w;
    const int m = (int)s[12];
    double2* C = work + off;
    double2* NT = work2 + off;
    double2* Tw = Tm + off;
    double2* D = DR + (long)w * M;
    const double2* Yw = Yin + off;
    double2* u0 = hh + (long)w * M;
    double* tau = htau + (long)w * M;

    for (long e = threadIdx.x; e < (long)M * m; e += nt) {
        int r = (int)(e / m), c = (int)(e % m);
        C[(long)r * M + c] = cmul(Yw[(long)r * M + c], D[c]);
    }
    __syncthreads();
    qrcp_panel(C, M, M, m, m, perm, cn, u0, tau, shv, shi, status);
    form_q(C, M, Qout + off, M, M, m, u0, tau);
    if (threadIdx.x == 0) {
        int k = m;
        for (int j = 0; j < m; ++j)
            if (sqrt(abs2(C[(long)j * M + j])) < thr) { k = j; break; }
        mnew = k < 1 ? 1 : k;
    }
    __syncthreads();
    const int mk = mnew;
    // new T rows i < m': sum_{j >= i} U_ij T[perm j][:], U = D^-1 R (unit upper)
    for (int col = threadIdx.x; col < M; col += nt) {
        for (int i = 0; i < mk; ++i) {
            const double2 dinv = cinv(C[(long)i * M + i]);
            double2 acc = Tw[(long)perm[i] * M + col];
            for (int j = i + 1; j < m; ++j)
                acc = cfma(cmul(C[(long)i * M + j], dinv), Tw[(long)perm[j] * M + col], acc);
            NT[(long)i * M + col] = acc;
        }
    }
    __syncthreads();
    for (long e = threadIdx.x; e < (long)mk * M; e += nt) Tw[e] = NT[e];
    for (int j = threadIdx.x; j < mk; j += nt) D[j] = C[(long)j * M + j];
    if (threadIdx.x == 0) s[12] = (double)mk;
}

// ---------------------------------------------------------------- Green's function
__global__ void __launch_bounds__(LR_THREADS) k_green_lr(const double2* __restrict__ Y, const double2* __restrict__ Tm,
                           const double2* __restrict__ DR, double2* __restrict__ work, double2* __restrict__ work2,
                           double2* __restrict__ z0, double2* __restrict__ z1, double2* __restrict__ G,
                           double2* __restrict__ hh, double* __restrict__ htau, const double* __restrict__ eps,
                           double* __restrict__ ws, int* __restrict__ status, int M, double lscale, double mu_T,
                           double thr, int constraint, int update, int with_gauss, double kdt) {
    extern __shared__ unsigned char smem_raw[];
    double2* ds = reinterpret_cast<double2*>(smem_raw);         // [M] d_s
    double2* invU = ds + M;                                     // [M] LU pivots^-1
    double* dl = reinterpret_cast<double*>(invU + M);           // [M] left block
    double* db = dl + M;                                        // [M] d_b
    double* cn = db + M;                                        // [M] column norms
    int* keepL = reinterpret_cast<int*>(cn + M);                // [M] L
    int* pivc = keepL + M;                                      // [M] pi_c
    int* lperm = pivc + M;                                      // [M] LU row order
    __shared__ double shv[32];
    __shared__ int shi[32];
    __shared__ double2 shc[32];
    __shared__ int sh_mL, nswap;
    const int w = blockIdx.x, nt = blockDim.x;
    const long off = (long)w * M * M;
    double* s = ws + (long)WSTRIDE * w;
    const int m = (int)s[12];
    const double2* Yw = Y + off;
    const double2* Tw = Tm + off;
    const double2* D = DR + (long)w * M;
    double2* C = work + off;      // core c, then r_c and U = d^-1 r_c
    double2* q = work2 + off;     // q = Y q_c      (M x m_T)
    double2* Qc = z0 + off;       // q_c (m x m_T), later Z = Mx^-1 d_s t (m_T x m_L)
    double2* Mx = z1 + off;       // d_b + d_s X, LU in place
    double2* Gw = G + off;
    double2* u0 = hh + (long)w * M;
    double* tau = htau + (long)w * M;

    for (int i = threadIdx.x; i < M; i += nt) dl[i] = exp(-lscale * (eps[i] - mu_T));
    __syncthreads();
    if (threadIdx.x == 0) {
        int n = 0, best = 0;
        for (int i = 0; i < M; ++i) {
            if (dl[i] >= thr) keepL[n++] = i;
            if (dl[i] > dl[best]) best = i;
        }
        if (n == 0) keepL[n++] = best;
        sh_mL = n;
        nswap = 0;
    }
    __syncthreads();
    const int mL = sh_mL;
    const int mT = m < mL ? m : mL;
    // core c[a][b] = D_a T[a][L_b] dl[L_b]
    for (long e = threadIdx.x; e < (long)m * mL; e += nt) {
        int a = (int)(e / mL), b = (int)(e % mL);
        C[(long)a * M + b] = cmul(D[a], Tw[(long)a * M + keepL[b]]) * dl[keepL[b]];
    }
    __syncthreads();
    qrcp_panel(C, M, m, mL, mT, pivc, cn, u0, tau, shv, shi, status);
    form_q(C, M, Qc, M, m, mT, u0, tau);
    // d = diag r_c and its split; U = d^-1 r_c (row i: columns i+1 .. m_L-1)
    for (int i = threadIdx.x; i < mT; i += nt) {
        const double2 d = C[(long)i * M + i];
        const double a = sqrt(abs2(d));
        if (a > 1.0) { db[i] = 1.0 / a; ds[i] = d * (1.0 / a); } else { db[i] = 1.0; ds[i] = d; }
    }
    __syncthreads();
    for (long e = threadIdx.x; e < (long)mT * mL; e += nt) {
        int i = (int)(e / mL), b = (int)(e % mL);
        if (b > i) C[(long)i * M + b] = cdiv(C[(long)i * M + b], C[(long)i * M + i]);
    }
    // q = Y[:, :m] q_c
    for (long e = threadIdx.x; e < (long)M * mT; e += nt) {
        int r = (int)(e / mT), c = (int)(e % mT);
        double2 acc = make_double2(0.0, 0.0);
        for (int a = 0; a < m; ++a) acc = cfma(Yw[(long)r * M + a], Qc[(long)a * M + c], acc);
        q[(long)r * M + c] = acc;
    }
    __syncthreads();
    // Mx = d_b + d_s X with X[i][l] = sum_{b >= i} U[i][b] q[L[pi_c b]][l]
    for (long e = threadIdx.x; e < (long)mT * mT; e += nt) {
        int i = (int)(e / mT), l = (int)(e % mT);
        double2 x = q[(long)keepL[pivc[i]] * M + l];
        for (int b = i + 1; b < mL; ++b) x = cfma(C[(long)i * M + b], q[(long)keepL[pivc[b]] * M + l], x);
        double2 v = cmul(ds[i], x);
        if (i == l) v.x += db[i];
        Mx[(long)i * M + l] = v;
    }
    for (int i = threadIdx.x; i < mT; i += nt) lperm[i] = i;
    __syncthreads();
    // LU of Mx with partial pivoting, in place
    for (int j = 0; j < mT; ++j) {
        double best = -1.0;
        int bidx = mT;
        for (int i = j + threadIdx.x; i < mT; i += nt) {
            double v = abs1(Mx[(long)i * M + j]);
            if (v > best) { best = v; bidx = i; }
        }
        int p = block_argmax(best, bidx, shv, shi);
        if (p >= mT) {
            p = j;
            if (threadIdx.x == 0) atomicOr(status, 1);
        }
        if (p != j) {
            for (int c = threadIdx.x; c < mT; c += nt) {
                double2 t = Mx[(long)j * M + c];
                Mx[(long)j * M + c] = Mx[(long)p * M + c];
                Mx[(long)p * M + c] = t;
            }
            if (threadIdx.x == 0) {
                int t = lperm[j]; lperm[j] = lperm[p]; lperm[p] = t;
                nswap ^= 1;
            }
        }
        __syncthreads();
        const double2 piv = Mx[(long)j * M + j];
        if (!(abs2(piv) > 0.0) && threadIdx.x == 0) atomicOr(status, 1);
        const double2 ip = cinv(piv);
        for (int i = j + 1 + threadIdx.x; i < mT; i += nt) Mx[(long)i * M + j] = cmul(Mx[(long)i * M + j], ip);
        if (threadIdx.x == 0) invU[j] = ip;
        __syncthreads();
        for (int c = j + 1 + threadIdx.x; c < mT; c += nt) {
            const double2 u = Mx[(long)j * M + c];
            for (int i = j + 1; i < mT; ++i) Mx[(long)i * M + c] = cfms(Mx[(long)i * M + j], u, Mx[(long)i * M + c]);
        }
        __syncthreads();
    }
    double2 ldm = make_double2(0.0, 0.0);
    double lsum = 0.0;
    for (int j = threadIdx.x; j < mT; j += nt) {
        ldm = ldm + clog(Mx[(long)j * M + j]);
        lsum += log(db[j]);
    }
    ldm = block_sum(ldm, shc);
    lsum = block_sum(lsum, shv);
    // Z = Mx^-1 (d_s U) column by column (column b of U has rows 0..min(b, m_T - 1))
    for (int b = threadIdx.x; b < mL; b += nt) {
        for (int j = 0; j < mT; ++j) {
            const int i = lperm[j];
            double2 v = i < b ? cmul(ds[i], C[(long)i * M + b]) : (i == b ? ds[i] : make_double2(0.0, 0.0));
            for (int k = 0; k < j; ++k) v = cfms(Mx[(long)j * M + k], Qc[(long)k * M + b], v);
            Qc[(long)j * M + b] = v;
        }
        for (int j = mT - 1; j >= 0; --j) {
            double2 v = Qc[(long)j * M + b];
            for (int k = j + 1; k < mT; ++k) v = cfms(Mx[(long)j * M + k], Qc[(long)k * M + b], v);
            Qc[(long)j * M + b] = cmul(v, invU[j]);
        }
    }
    __syncthreads();
    // G = I - q Z on the columns L[pi_c b]; identity elsewhere
    for (long e = threadIdx.x; e < (long)M * M; e += nt) {
        int r = (int)(e / M), c = (int)(e % M);
        Gw[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (long e = threadIdx.x; e < (long)M * mL; e += nt) {
        int r = (int)(e / mL), b = (int)(e % mL);
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < mT; ++i) acc = cfma(q[(long)r * M + i], Qc[(long)i * M + b], acc);
        const int c = keepL[pivc[b]];
        Gw[(long)r * M + c] = Gw[(long)r * M + c] - acc;
    }
    __syncthreads();
    double2 trg = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < M; i += nt) trg = trg + Gw[(long)i * M + i];
    trg = block_sum(trg, shc);
    if (threadIdx.x == 0) {
        double2 ld = ldm;
        ld.x -= lsum;
        ld.y += kPi * (double)nswap;
        if (!isfinite(ld.x) || !isfinite(ld.y)) atomicOr(status, 1);
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
                    s[8] += dlnS.x - tan(lnS.y) * dlnS.y;
                }
            }
        }
        s[3] = ld.x;
        s[4] = remainder(ld.y, 2.0 * kPi);
        s[9] = tk.x;
        s[10] = tk.y;
    }
}

int lr_threads(int M) {
    int t = ((M + 31) / 32) * 32;
    return t > LR_THREADS ? LR_THREADS : (t < 32 ? 32 : t);
}

}  // namespace

cudaError_t launch_qrcp_lr(ftq_ctx* c) {
    const int M = c->M;
    const size_t sm = (sizeof(double) + sizeof(int)) * M;
    {
        LaunchScope ls(c, FTQ_K_QRCP);
        k_qrcp_lr<<<c->W, lr_threads(M), sm, c->stream>>>(c->Y, c->zbuf[0], c->work, c->work2, c->DR, c->Tinv, c->hh,
                                                         c->htau, c->wstate, c->status, M, c->opts.low_rank_threshold);
    }
    double2* qn = c->zbuf[0];
    c->zbuf[0] = c->Y;
    c->Y = qn;
    return cudaGetLastError();
}

cudaError_t launch_green_lr(ftq_ctx* c, const double2* Y, int k, bool update, bool physical) {
    const int M = c->M;
    const size_t sm = (2 * sizeof(double2) + 3 * sizeof(double) + 3 * sizeof(int)) * M;
    static size_t sm_set = 0;
    if (sm > 48 * 1024 && sm > sm_set) {
        cudaError_t e = cudaFuncSetAttribute(k_green_lr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        sm_set = sm;
    }
    const double lscale = physical ? 0.0 : left_scale(c, k);
    LaunchScope ls(c, FTQ_K_GREEN);
    k_green_lr<<<c->W, lr_threads(M), sm, c->stream>>>(Y, c->Tinv, c->DR, c->work, c->work2, c->zbuf[0], c->zbuf[1],
                                                      c->G, c->hh, c->htau, c->tab.eps, c->wstate, c->status, M,
                                                      lscale, c->sys.mu_T, c->opts.low_rank_threshold,
                                                      c->opts.constraint, update ? 1 : 0, physical ? 0 : 1,
                                                      (double)k * c->sys.dtau);
    return cudaGetLastError();
}

}  // namespace ftq

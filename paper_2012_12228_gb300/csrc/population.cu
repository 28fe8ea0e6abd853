// Comb population control between slices (Computational Details: the comb
// method of Booth, Thom and Alavi, as described for CPMC-Lab), on the device.
//
// k_comb (one block): w_i = exp(ln|w_i| - max ln|w|) over alive walkers in
// parallel; then one thread forms the running sums C_i in index order in
// FP64, places the W teeth t_k = (k + xi) (S / W) (S = C_{W-1}), counts the
// copies n_i (walker i takes the teeth in [C_{i-1}, C_i), the last walker
// with a weight above 0 the rest), pairs the extra copies (ascending source) with the walkers that
// got none (ascending slot) and gives every surviving walker the weight S / W
// (ln|w| = ln(S / W) + max, phase 0).  k_copy_walkers then copies the whole
// walker state of each source into its destination slot; sources are
// survivors, destinations are not, so the copy is in place.
#include <cmath>

#include "ftq_internal.h"

namespace ftq {
namespace {

struct CopyPlan {
    double* base[8];      // per-walker buffers
    long words[8];        // 8-byte words per walker
    int n;
};

// wsc and cnt point to shared memory when the walkers fit (staged = true),
// else to global scratch; the arithmetic and its order are the same.
__global__ void k_comb(double* __restrict__ ws, double* __restrict__ wsc_g, int* __restrict__ cnt_g,
                       int* __restrict__ parent, int* __restrict__ pairs, int W, double xi,
                       int* __restrict__ status, bool staged) {
    __shared__ double shm[32];
    extern __shared__ unsigned char smem_raw[];
    double* wsc = staged ? reinterpret_cast<double*>(smem_raw) : wsc_g;
    int* cnt = staged ? reinterpret_cast<int*>(wsc + W) : cnt_g;
    const int tid = threadIdx.x, nt = blockDim.x;
    double m = -INFINITY;
    for (int i = tid; i < W; i += nt) {
        const double* s = ws + (long)WSTRIDE * i;
        if (s[2] > 0.5 && isfinite(s[0]) && s[0] > m) m = s[0];
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) shm[tid >> 5] = m;
    __syncthreads();
    double ref = shm[0];
    for (int i = 1; i < (nt + 31) / 32; ++i) ref = fmax(ref, shm[i]);
    if (!(ref > -INFINITY)) {                  // no walker alive: nothing to comb
        if (tid == 0) {
            atomicOr(status, 1);
            pairs[0] = 0;
        }
        for (int i = tid; i < W; i += nt) parent[i] = i;
        return;
    }
    for (int i = tid; i < W; i += nt) {
        const double* s = ws + (long)WSTRIDE * i;
        wsc[i] = (s[2] > 0.5 && isfinite(s[0])) ? exp(s[0] - ref) : 0.0;   // non-finite ln|w| weighs 0
    }
    __syncthreads();
    if (tid != 0) return;
    double S = 0.0;
    int last = 0;                              // the last walker with a weight above 0
    for (int i = 0; i < W; ++i) {
        S += wsc[i];
        if (wsc[i] > 0.0) last = i;
    }
    const double step = S / (double)W;
    int k = 0;
    double C = 0.0;
    for (int i = 0; i < W; ++i) {
        C += wsc[i];
        int n = 0;
        // teeth that rounding places at or beyond S go to the last walker
        // that carries weight, never to a dead one
        while (k < W && i <= last && (i == last || ((double)k + xi) * step < C)) {
            ++n;
            ++k;
        }
        cnt[i] = n;
    }
    int np = 0, e = 0;
    for (int i = 0; i < W; ++i)
        for (int c = 1; c < cnt[i]; ++c) {
            while (cnt[e] != 0) ++e;
            pairs[1 + np] = i;
            pairs[1 + W + np] = e;
            ++np;
            ++e;
        }
    pairs[0] = np;
    const double lw = log(S / (double)W) + ref;
    for (int i = 0; i < W; ++i) {
        parent[i] = cnt[i] > 0 ? i : -1;
        if (cnt[i] > 0) {
            double* s = ws + (long)WSTRIDE * i;
            s[0] = lw;
            s[1] = 0.0;
            s[2] = 1.0;
        }
    }
    for (int p = 0; p < np; ++p) parent[pairs[1 + W + p]] = pairs[1 + p];
}

// Pair branching (QWalk's method, which the paper uses for Theta <= 0.25),
// one block: u_i = w_i / (S / W) with S summed in index order by one thread;
// heavy walkers (u > 2) ranked by decreasing u and light ones (u < 1/2) by
// increasing u (ties to the lower index) in parallel; pair k = (k-th heavy a,
// k-th light b) keeps a when draws[k] < u_a / (u_a + u_b), else b; the kept
// walker gets weight (w_a + w_b) / 2 and is copied into the other slot.
__global__ void k_pair_branch(double* __restrict__ ws, const double* __restrict__ draws,
                              int* __restrict__ parent, int* __restrict__ pairs, int W, int* __restrict__ status) {
    __shared__ double shm[32];
    __shared__ double mean_sh;
    __shared__ int nh_sh, nl_sh;
    extern __shared__ unsigned char smem_raw[];
    double* wsc = reinterpret_cast<double*>(smem_raw);     // [W] scaled weights
    double* u = wsc + W;                                   // [W] weights over their mean
    int* heavy = reinterpret_cast<int*>(u + W);            // [W] heavy walker of rank r
    int* light = heavy + W;                                // [W] light walker of rank r
    const int tid = threadIdx.x, nt = blockDim.x;
    double m = -INFINITY;
    for (int i = tid; i < W; i += nt) {
        const double* s = ws + (long)WSTRIDE * i;
        if (s[2] > 0.5 && isfinite(s[0]) && s[0] > m) m = s[0];
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) shm[tid >> 5] = m;
    if (tid == 0) nh_sh = nl_sh = 0;
    __syncthreads();
    double ref = shm[0];
    for (int i = 1; i < (nt + 31) / 32; ++i) ref = fmax(ref, shm[i]);
    if (!(ref > -INFINITY)) {
        if (tid == 0) {
            atomicOr(status, 1);
            pairs[0] = 0;
        }
        for (int i = tid; i < W; i += nt) parent[i] = i;
        return;
    }
    for (int i = tid; i < W; i += nt) {
        const double* s = ws + (long)WSTRIDE * i;
        wsc[i] = (s[2] > 0.5 && isfinite(s[0])) ? exp(s[0] - ref) : 0.0;   // non-finite ln|w| weighs 0
    }
    __syncthreads();
    if (tid == 0) {
        double S = 0.0;
        for (int i = 0; i < W; ++i) S += wsc[i];
        mean_sh = S / (double)W;
    }
    __syncthreads();
    const double mean = mean_sh;
    for (int i = tid; i < W; i += nt) {
        u[i] = wsc[i] / mean;
        parent[i] = i;
    }
    __syncthreads();
    for (int i = tid; i < W; i += nt) {
        const double ui = u[i];
        if (ui > 2.0) {
            int r = 0;
            for (int j = 0; j < W; ++j) r += (u[j] > 2.0 && (u[j] > ui || (u[j] == ui && j < i))) ? 1 : 0;
            heavy[r] = i;
            atomicAdd(&nh_sh, 1);
        } else if (ui < 0.5) {
            int r = 0;
            for (int j = 0; j < W; ++j) r += (u[j] < 0.5 && (u[j] < ui || (u[j] == ui && j < i))) ? 1 : 0;
            light[r] = i;
            atomicAdd(&nl_sh, 1);
        }
    }
    __syncthreads();
    const int np = min(nh_sh, nl_sh);
    for (int k = tid; k < np; k += nt) {
        const int a = heavy[k], b = light[k];
        const bool keep_a = draws[k] < u[a] / (u[a] + u[b]);
        const int src = keep_a ? a : b, dst = keep_a ? b : a;
        double* s = ws + (long)WSTRIDE * src;
        s[0] = log(0.5 * (wsc[a] + wsc[b])) + ref;
        s[1] = 0.0;
        s[2] = 1.0;
        pairs[1 + k] = src;
        pairs[1 + W + k] = dst;
        parent[dst] = src;
    }
    if (tid == 0) pairs[0] = np;
}

__global__ void k_copy_walkers(const int* __restrict__ pairs, CopyPlan plan, int W) {
    const int p = blockIdx.y;
    if (p >= pairs[0]) return;
    const long src = pairs[1 + p], dst = pairs[1 + W + p];
    const long t0 = blockIdx.x * (long)blockDim.x + threadIdx.x, step = (long)gridDim.x * blockDim.x;
    for (int b = 0; b < plan.n; ++b) {
        const long n = plan.words[b];
        const double* s = plan.base[b] + n * src;
        double* d = plan.base[b] + n * dst;
        if ((n & 1) == 0) {           // 16-byte copies (buffers are 256-byte aligned, strides even)
            const double2* s2 = reinterpret_cast<const double2*>(s);
            double2* d2 = reinterpret_cast<double2*>(d);
            for (long i = t0; i < n / 2; i += step) d2[i] = s2[i];
        } else {
            for (long i = t0; i < n; i += step) d[i] = s[i];
        }
    }
}

}  // namespace

static CopyPlan walker_state_plan(ftq_ctx* c) {
    const long MM = (long)c->M * c->M;
    CopyPlan plan{};
    auto add = [&](void* p, long words) {
        if (p && plan.n < 8) {
            plan.base[plan.n] = static_cast<double*>(p);
            plan.words[plan.n] = words;
            ++plan.n;
        }
    };
    if (c->opts.precision == FTQ_FP64) {
        add(c->Y, 2 * MM);
    } else {
        add(c->Ypl, (long)c->LD * 2 * c->Kp);                 // two planes of LD x 2 Kp floats
        add(c->G32, MM);                                       // float2 = one word
        add(c->Yf, (long)c->LD * c->Kp);                       // one plane of LD x 2 Kp floats
    }
    add(c->Tinv, 2 * MM);
    add(c->G, 2 * MM);
    add(c->DR, 2L * c->M);
    add(c->wstate, WSTRIDE);
    return plan;
}

cudaError_t launch_population_control(ftq_ctx* c, double xi, int* parent_out) {
    const int W = c->W;
    const CopyPlan plan = walker_state_plan(c);
    {
        LaunchScope ls(c, FTQ_K_POPULATION);
        const size_t sm = (sizeof(double) + sizeof(int)) * (size_t)W;
        const bool staged = sm <= 96 * 1024;
        if (staged && sm > 48 * 1024)
            cudaFuncSetAttribute(k_comb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_comb<<<1, 256, staged ? sm : 0, c->stream>>>(c->wstate, c->pc_w, c->pc_cnt, c->pc_parent, c->pc_pairs,
                                                       W, xi, c->status, staged);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls(c, FTQ_K_POPULATION);
        k_copy_walkers<<<dim3(32, (unsigned)W), 256, 0, c->stream>>>(c->pc_pairs, plan, W);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && parent_out)
        e = cudaMemcpyAsync(parent_out, c->pc_parent, sizeof(int) * W, cudaMemcpyDeviceToDevice, c->stream);
    return e;
}

cudaError_t launch_pair_branch(ftq_ctx* c, const double* draws_host, int* parent_out) {
    const int W = c->W;
    const CopyPlan plan = walker_state_plan(c);
    // the draws go through the comb's weight scratch (W doubles >= W / 2 draws)
    cudaError_t e = cudaMemcpyAsync(c->pc_w, draws_host, sizeof(double) * (size_t)(W / 2), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) return e;
    const size_t sm = (2 * sizeof(double) + 2 * sizeof(int)) * (size_t)W;
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(k_pair_branch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    {
        LaunchScope ls(c, FTQ_K_POPULATION);
        k_pair_branch<<<1, 256, sm, c->stream>>>(c->wstate, c->pc_w, c->pc_parent, c->pc_pairs, W, c->status);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls(c, FTQ_K_POPULATION);
        k_copy_walkers<<<dim3(32, (unsigned)W), 256, 0, c->stream>>>(c->pc_pairs, plan, W);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && parent_out)
        e = cudaMemcpyAsync(parent_out, c->pc_parent, sizeof(int) * W, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);    // the host draws are read before return
    return e;
}

}  // namespace ftq

// C ABI of the walker-propagation library: context lifetime, device
// allocations, and the per-slice launch sequence.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ftq_internal.h"

namespace {

thread_local std::string g_init_error;

int fail(ftq_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg; else g_init_error = msg;
    return code;
}

int cuda_fail(ftq_ctx* c, cudaError_t e, const char* where) {
    cudaGetLastError();     // a non-sticky error must not be reported again by a later call
    return fail(c, FTQ_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t dalloc(ftq_ctx* c, T** p, size_t n) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * n);
    if (e == cudaSuccess) c->bytes += sizeof(T) * n;
    return e;
}

template <typename T>
cudaError_t upload(ftq_ctx* c, T** p, const std::vector<T>& v) {
    cudaError_t e = dalloc(c, p, v.size() ? v.size() : 1);
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

void free_all(ftq_ctx* c) {
    void* ptrs[] = {c->Y, c->Tinv, c->G, c->work, c->work2, c->zbuf[0], c->zbuf[1], c->DR, c->phi,
                    c->Ypl, c->zpl[0], c->zpl[1], c->G32, c->w32,
                    c->hh, c->htau, c->perm, c->wstate, c->est, c->red, c->status,
                    c->tab.vidx, c->tab.pair_ptr, c->tab.pair_a, c->tab.pair_b, c->tab.eps, c->tab.h,
                    c->tab.cq, c->tab.vq, c->tab.vqf, c->tab.ksq, c->tab.g0, c->items, c->tab.pk, c->tab.qcube,
                    c->tab.hf, c->phi32, c->xbuf, c->xsum, c->pc_w, c->pc_cnt, c->pc_parent, c->pc_pairs,
                    c->sq_walker, c->sq_w, c->sq_out, c->Yf, c->tab.eplus, c->trk, c->trk_out, c->items_lr};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// A member of a batch runs on the batch's private stream, while the caller
// hands in buffers that live on its own stream.  A call on a member that
// reads or writes caller device memory therefore waits for the caller's
// stream before its work and makes the caller's stream wait for that work
// after it.  Nothing happens for a stand-alone context (one stream).
struct CallerOrder {
    ftq_ctx* c;
    explicit CallerOrder(ftq_ctx* c_) : c(c_) { link(c->caller_stream, c->stream); }
    ~CallerOrder() { link(c->stream, c->caller_stream); }
    void link(cudaStream_t from, cudaStream_t to) {
        if (!c || !c->member) return;
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return;
        if (cudaEventRecord(ev, from) == cudaSuccess) cudaStreamWaitEvent(to, ev, 0);
        cudaEventDestroy(ev);
    }
};

}  // namespace

namespace ftq {
// Records a failure that is reported by ftq_last_error(NULL).
void set_global_error(const std::string& msg) { g_init_error = msg; }
}  // namespace ftq

extern "C" {

int ftq_init_ueg(ftq_ctx** out, int N, int M, double rs, double theta, double mu, double dtau,
                 const ftq_opts* opts) {
    if (!out || !opts) return fail(nullptr, FTQ_EINVAL, "out and opts must not be NULL");
    *out = nullptr;
    if (opts->walkers <= 0) return fail(nullptr, FTQ_EINVAL, "walkers must be positive");
    if (opts->exp_order < 1 || opts->exp_order > 32) return fail(nullptr, FTQ_EINVAL, "exp_order must be in 1..32");
    if (opts->stabilise_every < 0) return fail(nullptr, FTQ_EINVAL, "stabilise_every must be >= 0");
    if (opts->precision != FTQ_FP64 && opts->precision != FTQ_MIXED && opts->precision != FTQ_MIXED_SIMT &&
        opts->precision != FTQ_MIXED_F64UDT)
        return fail(nullptr, FTQ_EINVAL, "unknown precision");
    if (opts->constraint != FTQ_PHASELESS && opts->constraint != FTQ_FREE)
        return fail(nullptr, FTQ_EINVAL, "unknown constraint");
    if (opts->overlap != FTQ_OVERLAP_PAPER && opts->overlap != FTQ_OVERLAP_MODIFIED)
        return fail(nullptr, FTQ_EINVAL, "unknown overlap");
    if (opts->force_bias_cap != 0.0)
        return fail(nullptr, FTQ_EINVAL, "force_bias_cap must be 0: no force-bias cap is implemented");
    if (!(opts->low_rank_threshold >= 0.0) || !std::isfinite(opts->low_rank_threshold))
        return fail(nullptr, FTQ_EINVAL, "low_rank_threshold must be finite and >= 0");
    if (opts->low_rank_threshold > 0.0 && opts->precision == FTQ_MIXED_SIMT)
        return fail(nullptr, FTQ_EINVAL, "low-rank truncation runs with FTQ_FP64 or the tensor-core mixed path");
    if (N % 2 != 0) return fail(nullptr, FTQ_EINVAL, "N must be even (unpolarised gas)");
    ftq_ctx* c = new (std::nothrow) ftq_ctx();
    if (!c) return fail(nullptr, FTQ_ENOMEM, "host allocation failed");
    std::string why = ftq::build_ueg(c->sys, N, M, rs, theta, mu, dtau);
    if (!why.empty()) {
        delete c;
        return fail(nullptr, FTQ_EINVAL, why);
    }
    // the per-walker kernels loop over rows and columns with at most 1024
    // threads; their shared arrays grow with M (and with the number of
    // transfers): the complex128 path is checked up to M = 1189, the mixed
    // path up to M = 1021
    const int max_m = opts->precision == FTQ_FP64 ? 2047 : 1021;
    if (M > max_m) {
        delete c;
        return fail(nullptr, FTQ_EINVAL, "M = " + std::to_string(M) + " exceeds " + std::to_string(max_m) +
                                              " for this precision");
    }
    c->opts = *opts;
    c->stream = reinterpret_cast<cudaStream_t>(opts->cuda_stream);
    c->W = opts->walkers;
    c->M = M;
    c->nslot = 2 * c->sys.nq_half + 1;
    const size_t W = c->W, MM = (size_t)M * M;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (opts->precision == FTQ_FP64 || opts->low_rank_threshold > 0.0) {
        chk(dalloc(c, &c->Y, W * MM));      // the mixed low-rank path keeps a complex128 copy of the chain
    }
    if (opts->precision != FTQ_FP64) {
        c->Kp = (M + 15) / 16 * 16;       // 2 Kp is a whole number of 32-float k tiles
        c->LD = (M + 7) / 8 * 8;
        const size_t wsz = 2 * (size_t)c->LD * 2 * c->Kp;
        chk(dalloc(c, &c->Ypl, W * wsz));
        chk(dalloc(c, &c->Yf, W * wsz / 2));
        chk(dalloc(c, &c->zpl[0], W * wsz));
        chk(dalloc(c, &c->zpl[1], W * wsz));
        chk(dalloc(c, &c->G32, W * MM));
        // one allocation: the LU and solve halves for the QR and blocked LU
        // kernels, or per walker one contiguous M x 2M complex block for the
        // tensor-core Gauss-Jordan Green kernel
        chk(dalloc(c, &c->w32, W * std::max(2 * MM, (ftq::green_tc_floats(M) + 1) / 2)));
        c->w2_32 = c->w32 + W * MM;
        chk(dalloc(c, &c->xsum, W * MM));
    }
    chk(dalloc(c, &c->Tinv, W * MM));
    chk(dalloc(c, &c->G, W * MM));
    chk(dalloc(c, &c->work, W * MM));
    chk(dalloc(c, &c->work2, W * MM));
    chk(dalloc(c, &c->zbuf[0], W * MM));
    chk(dalloc(c, &c->zbuf[1], W * MM));
    chk(dalloc(c, &c->DR, W * M));
    chk(dalloc(c, &c->phi, W * c->nslot));
    if (e == cudaSuccess) chk(cudaMemset(c->phi, 0, sizeof(double2) * W * c->nslot));
    if (opts->precision != FTQ_FP64) {
        chk(dalloc(c, &c->phi32, W * c->nslot));
        if (e == cudaSuccess) chk(cudaMemset(c->phi32, 0, sizeof(float2) * W * c->nslot));
    }
    chk(dalloc(c, &c->hh, W * M));
    chk(dalloc(c, &c->htau, W * M));
    chk(dalloc(c, &c->perm, W * M));
    chk(dalloc(c, &c->wstate, W * ftq::WSTRIDE));
    chk(dalloc(c, &c->pc_w, W));
    chk(dalloc(c, &c->pc_cnt, W));
    chk(dalloc(c, &c->pc_parent, W));
    chk(dalloc(c, &c->pc_pairs, 1 + 2 * W));
    chk(dalloc(c, &c->est, W * ftq::WSTRIDE));
    chk(dalloc(c, &c->red, 16));
    chk(dalloc(c, &c->status, 1));
    const ftq::UegSetup& s = c->sys;
    std::vector<double> h(M), ksq(M), g0(M);
    for (int i = 0; i < M; ++i) {
        h[i] = std::exp(-0.5 * s.dtau * (s.eps[i] + s.deps[i] - s.mu));
        ksq[i] = 2.0 * s.eps[i];
        g0[i] = 1.0 / (1.0 + std::exp(-s.beta * (s.eps[i] - s.mu_T)));
    }
    if (e == cudaSuccess) {
        chk(upload(c, &c->tab.vidx, s.vidx));
        chk(upload(c, &c->tab.pair_ptr, s.pair_ptr));
        chk(upload(c, &c->tab.pair_a, s.pair_a));
        chk(upload(c, &c->tab.pair_b, s.pair_b));
        chk(upload(c, &c->tab.eps, s.eps));
        chk(upload(c, &c->tab.h, h));
        chk(upload(c, &c->tab.cq, s.cq));
        chk(upload(c, &c->tab.vq, s.vq));
        {
            std::vector<float2> vqf(s.vq.size());
            for (size_t q = 0; q < s.vq.size(); ++q) {
                vqf[q].x = (float)s.vq[q];
                vqf[q].y = (float)(s.vq[q] - (double)vqf[q].x);
            }
            chk(upload(c, &c->tab.vqf, vqf));
        }
        chk(upload(c, &c->tab.ksq, ksq));
        chk(upload(c, &c->tab.g0, g0));
        chk(upload(c, &c->tab.pk, s.pk));
        std::vector<float2> hf(M);
        for (int i = 0; i < M; ++i) {
            hf[i].x = (float)h[i];
            hf[i].y = (float)(h[i] - (double)hf[i].x);
        }
        chk(upload(c, &c->tab.hf, hf));
        chk(upload(c, &c->tab.qcube, s.qcube));
        // exchange work units: chunks of 32 pairs of every odd (+Q) slot
        std::vector<int4> eplus;
        for (int sl = 1; sl < c->nslot; sl += 2)
            for (int e = s.pair_ptr[sl]; e < s.pair_ptr[sl + 1]; e += 32)
                eplus.push_back(make_int4(s.pair_ptr[sl], s.pair_ptr[sl + 1], e, (sl - 1) >> 1));
        c->tab.neplus = (int)eplus.size();
        chk(upload(c, &c->tab.eplus, eplus));
    }
    if (e == cudaSuccess && (opts->precision == FTQ_MIXED || opts->precision == FTQ_MIXED_F64UDT)) {
        if (!ftq::tc_supported(M)) {
            free_all(c);
            delete c;
            return fail(nullptr, FTQ_ECUDA, "the driver does not expose cuTensorMapEncodeTiled");
        }
        chk(ftq::tc_make_maps(c));
    }
    if (e == cudaSuccess) chk(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    if (e == cudaSuccess) chk(ftq::launch_init_walkers(c));
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? FTQ_ENOMEM : FTQ_ECUDA;
        std::string msg = std::string("device setup failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_all(c);
        delete c;
        return fail(nullptr, code, msg);
    }
    *out = c;
    return FTQ_OK;
}

int ftq_reset(ftq_ctx* c) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    c->resampled = false;
    c->trk_n = 0;
    if (c->items_lr) {                 // every walker is back at full rank
        cudaFree(c->items_lr);
        c->items_lr = nullptr;
    }
    cudaError_t e = ftq::launch_init_walkers(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "reset");
    return FTQ_OK;
}

int ftq_propagate_slices(ftq_ctx* c, int n_slices, const double* fields_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    CallerOrder order(c);
    if (n_slices < 0) return fail(c, FTQ_EINVAL, "n_slices must be >= 0");
    if (c->k + n_slices > c->sys.n_slices)
        return fail(c, FTQ_EINVAL, "propagation would pass tau = beta; call ftq_reset first");
    const size_t per_slice = (size_t)c->W * c->sys.n_alpha;
    if (n_slices > 0 && !fields_dev && !c->xbuf) {
        cudaError_t e = cudaMalloc(&c->xbuf, per_slice * sizeof(double));
        if (e != cudaSuccess) {
            c->xbuf = nullptr;
            return cuda_fail(c, e, "field buffer");
        }
        c->bytes += per_slice * sizeof(double);
    }
    for (int t = 0; t < n_slices; ++t) {
        const int k = c->k + 1;
        const double* x = fields_dev ? fields_dev + per_slice * t : c->xbuf;
        cudaError_t e = cudaSuccess;
        if (!fields_dev) {
            ftq::LaunchScope ls(c, FTQ_K_FIELDS);
            e = ftq::launch_philox_fields(c->xbuf, c->opts.seed, 0u, k - 1, 1, c->W, c->sys.n_alpha, c->stream);
        }
        if (e == cudaSuccess) e = ftq::launch_force_bias(c, x);
        if (e == cudaSuccess) e = ftq::launch_chain(c);
        if (e == cudaSuccess && c->opts.stabilise_every > 0 && k % c->opts.stabilise_every == 0)
            e = ftq::launch_qrcp(c);
        if (e == cudaSuccess) e = ftq::launch_green(c, k, true);
        if (e == cudaSuccess && c->track_every > 0 && k % c->track_every == 0) e = ftq::launch_slice_estimate(c, k);
        if (e != cudaSuccess) return cuda_fail(c, e, "propagate");
        c->k = k;
    }
    return FTQ_OK;
}

int ftq_fields(ftq_ctx* c, int first_slice, int n_slices, double* out_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    CallerOrder order(c);
    if (!out_dev) return fail(c, FTQ_EINVAL, "out_dev must not be NULL");
    if (first_slice < 0 || n_slices < 0 || first_slice + n_slices > c->sys.n_slices)
        return fail(c, FTQ_EINVAL, "slice window outside [0, n)");
    ftq::LaunchScope ls(c, FTQ_K_FIELDS);
    cudaError_t e = ftq::launch_philox_fields(out_dev, c->opts.seed, 0u, first_slice, n_slices, c->W,
                                              c->sys.n_alpha, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fields");
    return FTQ_OK;
}

// The structure factor and the mu derivative keep two tables over every
// transfer in shared memory (32 bytes per slot).
static bool slot_tables_fit(const ftq_ctx* c) { return 2 * sizeof(double2) * (size_t)c->nslot <= 227 * 1024; }

int ftq_structure_factor(ftq_ctx* c, double* out_host, void* per_walker_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    if (!slot_tables_fit(c)) return fail(c, FTQ_EINVAL, "too many momentum transfers for the structure factor kernel");
    CallerOrder order(c);
    if (!out_host) return fail(c, FTQ_EINVAL, "out_host must not be NULL");
    if (!c->members.empty()) return fail(c, FTQ_EINVAL, "evaluate the members of a batch one by one");
    cudaError_t e = ftq::launch_structure_factor(c, static_cast<double*>(per_walker_dev));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, c->sq_out, sizeof(double) * (4 + 2 * (size_t)(c->nslot - 1)),
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "structure factor");
    return FTQ_OK;
}

int ftq_pair_branch(ftq_ctx* c, const double* draws_host, int* parent_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    CallerOrder order(c);
    if (!draws_host) return fail(c, FTQ_EINVAL, "draws_host must not be NULL");
    if (!c->members.empty()) return fail(c, FTQ_EINVAL, "branch the members of a batch one by one");
    if (c->opts.constraint == FTQ_FREE) return fail(c, FTQ_EINVAL, "pair branching acts on phaseless weights");
    if (c->W > 8192) return fail(c, FTQ_EINVAL, "pair branching holds at most 8192 walkers");
    for (int k = 0; k < c->W / 2; ++k)
        if (!(draws_host[k] >= 0.0 && draws_host[k] < 1.0)) return fail(c, FTQ_EINVAL, "draws must lie in [0, 1)");
    cudaError_t e = ftq::launch_pair_branch(c, draws_host, parent_dev);
    // copied walkers carry their ranks: the rank-compacted chain work list follows
    if (e == cudaSuccess && c->items_lr) e = ftq::tc_items_by_rank(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "pair branching");
    c->resampled = true;
    return FTQ_OK;
}

int ftq_population_control(ftq_ctx* c, double xi, int* parent_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    CallerOrder order(c);
    if (!c->members.empty()) return fail(c, FTQ_EINVAL, "comb the members of a batch one by one");
    if (!(xi >= 0.0 && xi < 1.0)) return fail(c, FTQ_EINVAL, "xi must lie in [0, 1)");
    if (c->opts.constraint == FTQ_FREE) return fail(c, FTQ_EINVAL, "the comb acts on phaseless weights");
    if (c->W > 65535) return fail(c, FTQ_EINVAL, "at most 65535 walkers");
    cudaError_t e = ftq::launch_population_control(c, xi, parent_dev);
    if (e == cudaSuccess && c->items_lr) e = ftq::tc_items_by_rank(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "population control");
    c->resampled = true;
    return FTQ_OK;
}

int ftq_stabilise(ftq_ctx* c) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    cudaError_t e = ftq::launch_qrcp(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "stabilise");
    return FTQ_OK;
}

int ftq_green(ftq_ctx* c, void* G_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    CallerOrder order(c);
    if (!G_dev) return fail(c, FTQ_EINVAL, "G_dev must not be NULL");
    cudaError_t e = ftq::launch_copy_green(c, reinterpret_cast<double2*>(G_dev));
    if (e != cudaSuccess) return cuda_fail(c, e, "green");
    return FTQ_OK;
}

int ftq_estimators(ftq_ctx* c, double* out_host, double* per_walker_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    CallerOrder order(c);
    if (!out_host) return fail(c, FTQ_EINVAL, "out_host must not be NULL");
    cudaError_t e = ftq::launch_estimators(c, per_walker_dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, c->red, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "estimators");
    return FTQ_OK;
}

int ftq_track_estimates(ftq_ctx* c, int every) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    if (every < 0) return fail(c, FTQ_EINVAL, "every must be >= 0");
    if (!c->members.empty()) return fail(c, FTQ_EINVAL, "track the members of a batch one by one");
    if (every > 0 && !c->trk) {
        const size_t rows = (size_t)c->sys.n_slices;
        cudaError_t e = dalloc(c, &c->trk, 8 * rows);
        if (e == cudaSuccess) e = dalloc(c, &c->trk_out, 8 * (rows + 1));
        if (e != cudaSuccess) {
            if (c->trk) cudaFree(c->trk);
            c->trk = nullptr;
            return fail(c, e == cudaErrorMemoryAllocation ? FTQ_ENOMEM : FTQ_ECUDA, "slice estimate record");
        }
    }
    c->track_every = every;
    return FTQ_OK;
}

int ftq_slice_estimates(ftq_ctx* c, double* out_host, int capacity) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    if (!out_host || capacity < 0) return fail(c, FTQ_EINVAL, "out_host must not be NULL and capacity >= 0");
    if (!c->trk) return fail(c, FTQ_EINVAL, "no slice estimates recorded: call ftq_track_estimates first");
    const int rows = c->trk_n < capacity ? c->trk_n : capacity;
    cudaError_t e = ftq::launch_slice_summary(c, c->trk_out, rows);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, c->trk_out, sizeof(double) * 8 * (size_t)(rows + 1), cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "slice estimates");
    return FTQ_OK;
}

int ftq_mu_grad(ftq_ctx* c, double* out_host, double* per_walker_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    if (!slot_tables_fit(c)) return fail(c, FTQ_EINVAL, "too many momentum transfers for the mu-derivative kernel");
    CallerOrder order(c);
    if (!out_host) return fail(c, FTQ_EINVAL, "out_host must not be NULL");
    if (c->k != c->sys.n_slices)
        return fail(c, FTQ_EINVAL, "the mu derivative is accumulated over a whole path: propagate to tau = beta first");
    if (c->resampled)
        return fail(c, FTQ_EINVAL, "the mu derivative at fixed draws is undefined across population control");
    cudaError_t e = ftq::launch_mu_grad(c, per_walker_dev);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, c->red + 8, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mu_grad");
    return FTQ_OK;
}

int ftq_weights(ftq_ctx* c, double* out_dev) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    CallerOrder order(c);
    if (!out_dev) return fail(c, FTQ_EINVAL, "out_dev must not be NULL");
    cudaError_t e = cudaMemcpy2DAsync(out_dev, sizeof(double) * 8, c->wstate, sizeof(double) * ftq::WSTRIDE,
                                      sizeof(double) * 8, c->W, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "weights");
    return FTQ_OK;
}

int ftq_ranks(ftq_ctx* c, int* ranks_host) {
    if (!c || !ranks_host) return fail(c, FTQ_EINVAL, "NULL argument");
    std::vector<double> r((size_t)c->W);
    cudaError_t e = cudaMemcpy2DAsync(r.data(), sizeof(double), c->wstate + 12, sizeof(double) * ftq::WSTRIDE,
                                      sizeof(double), c->W, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ranks");
    for (int w = 0; w < c->W; ++w) ranks_host[w] = (int)r[(size_t)w];
    return FTQ_OK;
}

int ftq_status(ftq_ctx* c, int* status_host) {
    if (!c || !status_host) return fail(c, FTQ_EINVAL, "NULL argument");
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "status");
    *status_host = (v & 2) ? FTQ_ETIMEOUT : (v ? FTQ_ENUMERIC : FTQ_OK);
    return FTQ_OK;
}

int ftq_set_green_kernel(ftq_ctx* c, int kind) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    if (kind < 0 || kind > 2) return fail(c, FTQ_EINVAL, "green kernel must be 0, 1 or 2");
    c->green_kind = kind;
    return FTQ_OK;
}

int ftq_set_wait_limit(ftq_ctx* c, int64_t polls) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    if (polls < -1) return fail(c, FTQ_EINVAL, "polls must be >= -1");
    c->wait_limit = polls;
    return FTQ_OK;
}

int ftq_query(const ftq_ctx* c, int key, int64_t* value) {
    if (!c || !value) return fail(const_cast<ftq_ctx*>(c), FTQ_EINVAL, "NULL argument");
    switch (key) {
        case FTQ_Q_M: *value = c->M; break;
        case FTQ_Q_N_ALPHA: *value = c->sys.n_alpha; break;
        case FTQ_Q_N_SLICES: *value = c->sys.n_slices; break;
        case FTQ_Q_SLICE: *value = c->k; break;
        case FTQ_Q_WALKERS: *value = c->W; break;
        case FTQ_Q_NCUT2: *value = c->sys.ncut2; break;
        case FTQ_Q_PRECISION: *value = c->opts.precision; break;
        case FTQ_Q_DEVICE_BYTES: *value = (int64_t)c->bytes; break;
        case FTQ_Q_QR_PANEL: *value = c->qr_nb; break;
        case FTQ_Q_GREEN_KERNEL:
            *value = (c->opts.precision == FTQ_FP64 || c->opts.low_rank_threshold > 0.0) ? 0
                     : (ftq::green_uses_tc(c) ? 1 : 2);
            break;
        default: return fail(const_cast<ftq_ctx*>(c), FTQ_EINVAL, "unknown query key");
    }
    return FTQ_OK;
}

int ftq_query_f64(const ftq_ctx* c, int key, double* value) {
    if (!c || !value) return fail(const_cast<ftq_ctx*>(c), FTQ_EINVAL, "NULL argument");
    switch (key) {
        case FTQ_F_BETA: *value = c->sys.beta; break;
        case FTQ_F_DTAU: *value = c->sys.dtau; break;
        case FTQ_F_MU: *value = c->sys.mu; break;
        case FTQ_F_MU_T: *value = c->sys.mu_T; break;
        case FTQ_F_L: *value = c->sys.L; break;
        case FTQ_F_E_M: *value = c->sys.E_M; break;
        default: return fail(const_cast<ftq_ctx*>(c), FTQ_EINVAL, "unknown query key");
    }
    return FTQ_OK;
}

int ftq_basis(const ftq_ctx* c, int32_t* nvec_host) {
    if (!c || !nvec_host) return fail(const_cast<ftq_ctx*>(c), FTQ_EINVAL, "NULL argument");
    for (size_t i = 0; i < c->sys.nvec.size(); ++i) nvec_host[i] = c->sys.nvec[i];
    return FTQ_OK;
}

int ftq_transfers(const ftq_ctx* c, int32_t* q_host) {
    if (!c || !q_host) return fail(const_cast<ftq_ctx*>(c), FTQ_EINVAL, "NULL argument");
    for (size_t i = 0; i < c->sys.qhalf.size(); ++i) q_host[i] = c->sys.qhalf[i];
    return FTQ_OK;
}

int ftq_profile(ftq_ctx* c, int enable) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    if (enable) {
        for (auto& sp : c->spans) { c->event_pool.push_back(sp.a); c->event_pool.push_back(sp.b); }
        c->spans.clear();
        for (int k = 0; k < FTQ_K_COUNT; ++k) { c->prof_ms[k] = 0; c->prof_n[k] = 0; }
    }
    c->prof = enable != 0;
    return FTQ_OK;
}

int ftq_profile_read(ftq_ctx* c, double* ms_host, int64_t* launches_host) {
    if (!c) return fail(nullptr, FTQ_EINVAL, "ctx is NULL");
    cudaError_t e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "profile_read");
    for (auto& sp : c->spans) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, sp.a, sp.b);
        if (e != cudaSuccess) return cuda_fail(c, e, "profile_read elapsed");
        c->prof_ms[sp.kind] += ms;
        c->prof_n[sp.kind] += 1;
        c->event_pool.push_back(sp.a);
        c->event_pool.push_back(sp.b);
    }
    c->spans.clear();
    for (int k = 0; k < FTQ_K_COUNT; ++k) {
        if (ms_host) ms_host[k] = c->prof_ms[k];
        if (launches_host) launches_host[k] = c->launches[k];
    }
    return FTQ_OK;
}

const char* ftq_last_error(const ftq_ctx* c) {
    if (!c) return g_init_error.c_str();
    return c->err.c_str();
}

void ftq_destroy(ftq_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    for (ftq_ctx* m : c->members) ftq_destroy(m);
    c->members.clear();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->owns_stream && c->stream) cudaStreamDestroy(c->stream);
    for (auto& sp : c->spans) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
    for (auto ev : c->event_pool) cudaEventDestroy(ev);
    free_all(c);
    delete c;
}

}  // extern "C"

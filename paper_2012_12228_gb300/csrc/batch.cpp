// Ragged batch of UEG systems: several (N, M) systems of different basis
// size propagated together.  Every Horner step of the tensor-core chain runs
// as ONE persistent launch over the work items of all systems; the launches
// of a propagation call are captured into a CUDA graph and replayed as one
// graph launch; the column tiling of each system's chain is autotuned.
#include <cmath>
#include <string>

#include "ftq_internal.h"

namespace ftq {
void set_global_error(const std::string& msg);
}

namespace {

int bfail(ftq_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg; else ftq::set_global_error(msg);
    return code;
}

// The slice loop of a batch: per slice force bias for every member, the p
// Horner steps as batched tensor-core launches, then QRCP / G per member.
cudaError_t run_slices(ftq_ctx* b, int n, const double* const* fields) {
    const int ns = (int)b->members.size();
    const int p = b->opts.exp_order, stab = b->opts.stabilise_every;
    for (int t = 0; t < n; ++t) {
        for (int s = 0; s < ns; ++s) {
            ftq_ctx* m = b->members[s];
            cudaError_t e = ftq::launch_force_bias(m, fields[s] + (size_t)t * m->W * m->sys.n_alpha);
            if (e != cudaSuccess) return e;
        }
        const float* zin[8];
        float* out[8];
        int cur = 0;
        for (int s = 0; s < ns; ++s) zin[s] = b->members[s]->Ypl;
        for (int j = p; j >= 1; --j) {
            for (int s = 0; s < ns; ++s) out[s] = b->members[s]->zpl[cur];
            cudaError_t e = ftq::tc_chain_step_batch(b, zin, out, j, p);
            if (e != cudaSuccess) return e;
            for (int s = 0; s < ns; ++s) zin[s] = out[s];
            cur ^= 1;
        }
        for (int s = 0; s < ns; ++s) {
            ftq_ctx* m = b->members[s];
            float* res = m->zpl[cur ^ 1];
            m->zpl[cur ^ 1] = m->Ypl;
            m->Ypl = res;
        }
        for (int s = 0; s < ns; ++s) {
            ftq_ctx* m = b->members[s];
            const int k = m->k + 1;
            cudaError_t e = cudaSuccess;
            if (stab > 0 && k % stab == 0) e = ftq::launch_qrcp(m);
            if (e == cudaSuccess) e = ftq::launch_green(m, k, true);
            if (e != cudaSuccess) return e;
            m->k = k;
        }
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int ftq_init_batch(ftq_ctx** out, int nsys, const ftq_system* systems, const ftq_opts* opts) {
    if (!out || !systems || !opts) return bfail(nullptr, FTQ_EINVAL, "NULL argument");
    *out = nullptr;
    if (nsys < 1 || nsys > 8) return bfail(nullptr, FTQ_EINVAL, "a batch holds 1 to 8 systems");
    if (opts->precision != FTQ_MIXED)
        return bfail(nullptr, FTQ_EINVAL, "a ragged batch runs the mixed-precision tensor-core path (FTQ_MIXED)");
    if (opts->low_rank_threshold != 0.0)
        return bfail(nullptr, FTQ_EINVAL, "a ragged batch runs at full rank");
    ftq_ctx* b = new ftq_ctx();
    b->opts = *opts;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->owns_stream = e == cudaSuccess;
    if (e != cudaSuccess) {
        delete b;
        return bfail(nullptr, FTQ_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    for (int s = 0; s < nsys; ++s) {
        ftq_opts o = *opts;
        o.walkers = systems[s].walkers;
        o.cuda_stream = b->stream;
        ftq_ctx* m = nullptr;
        int rc = ftq_init_ueg(&m, systems[s].N, systems[s].M, systems[s].rs, systems[s].theta, systems[s].mu,
                              systems[s].dtau, &o);
        if (rc != FTQ_OK) {
            std::string why = std::string("system ") + std::to_string(s) + ": " + ftq_last_error(nullptr);
            ftq_destroy(b);
            return bfail(nullptr, rc, why);
        }
        m->member = true;
        m->caller_stream = reinterpret_cast<cudaStream_t>(opts->cuda_stream);
        b->members.push_back(m);
    }
    e = ftq::tc_batch_items(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        ftq_destroy(b);
        return bfail(nullptr, FTQ_ECUDA, std::string("batch setup: ") + cudaGetErrorString(e));
    }
    *out = b;
    return FTQ_OK;
}

int ftq_batch_member(ftq_ctx* b, int s, ftq_ctx** member) {
    if (!b || !member) return bfail(b, FTQ_EINVAL, "NULL argument");
    if (s < 0 || s >= (int)b->members.size()) return bfail(b, FTQ_EINVAL, "no such member system");
    *member = b->members[s];
    return FTQ_OK;
}

int ftq_batch_propagate(ftq_ctx* b, int n_slices, const double* const* fields_dev) {
    if (!b || b->members.empty()) return bfail(b, FTQ_EINVAL, "not a batch context");
    if (n_slices < 0 || (n_slices > 0 && !fields_dev)) return bfail(b, FTQ_EINVAL, "bad fields or slice count");
    for (size_t s = 0; s < b->members.size(); ++s) {
        ftq_ctx* m = b->members[s];
        if (m->k + n_slices > m->sys.n_slices)
            return bfail(b, FTQ_EINVAL, "member " + std::to_string(s) + " would pass tau = beta");
        if (n_slices > 0 && !fields_dev[s]) return bfail(b, FTQ_EINVAL, "NULL fields for a member");
        if (m->prof) b->use_graph = false;   // per-launch event timing is not captured
    }
    if (n_slices == 0) return FTQ_OK;
    // order the batch stream after the caller's stream
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(b->opts.cuda_stream);
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
    if (e != cudaSuccess) return bfail(b, FTQ_ECUDA, std::string("stream order: ") + cudaGetErrorString(e));
    if (b->use_graph) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        cudaError_t er = e == cudaSuccess ? run_slices(b, n_slices, fields_dev) : e;
        cudaError_t ec = e == cudaSuccess ? cudaStreamEndCapture(b->stream, &graph) : e;
        e = er != cudaSuccess ? er : ec;
        if (e == cudaSuccess && b->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(b->gexec, graph, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
        }
        if (e == cudaSuccess && !b->gexec) e = cudaGraphInstantiate(&b->gexec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->gexec, b->stream);
        if (graph) cudaGraphDestroy(graph);
    } else {
        e = run_slices(b, n_slices, fields_dev);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return bfail(b, FTQ_ECUDA, std::string("batch propagate: ") + cudaGetErrorString(e));
    return FTQ_OK;
}

int ftq_autotune(ftq_ctx* c, int* choice, float* ms) {
    if (!c) return bfail(nullptr, FTQ_EINVAL, "ctx is NULL");
    std::vector<ftq_ctx*> targets = c->members.empty() ? std::vector<ftq_ctx*>{c} : c->members;
    for (size_t s = 0; s < targets.size(); ++s) {
        ftq_ctx* m = targets[s];
        if (m->opts.precision != FTQ_MIXED && m->opts.precision != FTQ_MIXED_F64UDT) {
            if (choice) choice[s] = 0;
            if (ms) ms[s] = 0.f;
            continue;
        }
        int best = 1;
        float bms = 0.f;
        cudaError_t e = ftq::tc_autotune(m, &best, &bms);
        int qnb = 0;
        float qms = 0.f;
        if (e == cudaSuccess) e = ftq::qr_autotune(m, &qnb, &qms);
        float gtc = 0.f, glu = 0.f;
        if (e == cudaSuccess) e = ftq::green_autotune(m, &gtc, &glu);
        if (e != cudaSuccess) return bfail(c, FTQ_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
        if (choice) choice[s] = best;
        if (ms) ms[s] = bms;
    }
    if (!c->members.empty()) {
        cudaError_t e = ftq::tc_batch_items(c);
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        if (e != cudaSuccess) return bfail(c, FTQ_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    }
    return FTQ_OK;
}

}  // extern "C"

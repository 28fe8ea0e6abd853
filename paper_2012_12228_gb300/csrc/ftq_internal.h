// Internal declarations shared by the host orchestrator and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "ftq.h"

namespace ftq {

// Per-walker state record, WSTRIDE doubles:
//   [0] ln|w|  [1] arg w  [2] alive  [3] Re ln det(I+A)  [4] Im ln det
//   [5] Re gauss_k  [6] Im gauss_k  [7] parity of det T
//   [8] d ln|w|/dmu  [9] Re t_k  [10] Im t_k  (t_k = d ln det(I+A_k)/dmu)
//   [11] d arg w/dmu  [12] rank m of the right block (M at full rank)  [13..15] unused
// The per-walker estimator record uses the same stride:
//   [0..2] as above, [3] Re E, [4] Im E, [5] Re N, [6] Im N, [7] unused,
//   [8] d ln|w|/dmu, [9] d arg w/dmu, [10] Re dE, [11] Im dE, [12] Re dN, [13] Im dN
constexpr int WSTRIDE = 16;

// Static description of one UEG system (Sec. "Uniform Electron Gas" and
// "Computational Details").  Built on the host once per context.
struct UegSetup {
    int N = 0, M = 0, ncut2 = 0, R = 0;       // R = isqrt(ncut2)
    int nq_half = 0, n_alpha = 0, n_slices = 0;
    double rs = 0, theta = 0, L = 0, Omega = 0, TF = 0, beta = 0, dtau = 0;
    double mu = 0, mu_T = 0, E_M = 0;
    std::vector<int> nvec;        // [M][3]
    std::vector<int> qhalf;       // [nq_half][3]
    std::vector<double> eps;      // |K|^2 / 2
    std::vector<double> deps;     // one-body correction of the sum-of-squares form
    std::vector<double> cq;       // sqrt(2 pi / (Omega Q^2)), half space
    std::vector<double> vq;       // 4 pi / (Omega Q^2), half space
    // slot of the phi table addressed by (K', K): 0 for K' == K, 1 + 2q for
    // K' - K = +Q_q, 2 + 2q for K' - K = -Q_q.
    std::vector<uint16_t> vidx;   // [M][M]
    // slot of a difference vector: V[i][k] = phi[qcube[pk[i] - pk[k] + qoff]]
    // with pk[i] = nx S^2 + ny S + nz and S = 4 R + 1 (the cube of all
    // differences of two basis vectors)
    int qS = 0, qoff = 0;
    std::vector<int> pk;          // [M]
    std::vector<uint16_t> qcube;  // [S^3]
    // pairs (a, b) with n_a - n_b = Q for every slot, CSR by slot
    std::vector<int> pair_ptr;    // [2 nq_half + 2]
    std::vector<int> pair_a, pair_b;
};

// Returns an empty string on success, else the reason.
std::string build_ueg(UegSetup& s, int N, int M, double rs, double theta, double mu, double dtau);

// Device-side constant tables.
struct DevTables {
    uint16_t* vidx = nullptr;     // [M][M]
    int* pair_ptr = nullptr;      // [nslot + 1]
    int* pair_a = nullptr;
    int* pair_b = nullptr;
    double* eps = nullptr;        // [M]
    double* h = nullptr;          // exp(-dtau/2 (eps + deps - mu)) [M]
    double* cq = nullptr;         // [nq_half]
    double* vq = nullptr;         // [nq_half]
    float2* vqf = nullptr;        // [nq_half] v_Q as a float pair (hi, lo)
    double* ksq = nullptr;        // |K|^2 [M]
    double* g0 = nullptr;         // diagonal of G(0) = (I + B_T^n)^-1 [M]
    int* pk = nullptr;            // packed basis coordinates [M]
    float2* hf = nullptr;         // h as float pairs (hi, lo) [M]
    uint16_t* qcube = nullptr;    // difference -> slot [S^3]
    int4* eplus = nullptr;        // exchange work units: per half-space transfer (odd slot) and chunk
                                  // of 32 of its pairs, {first, end of the slot's pair list, first pair
                                  // of the chunk, index into v_Q}
    int neplus = 0;
};

}  // namespace ftq

struct ftq_ctx {
    ftq::UegSetup sys;
    ftq::DevTables tab;
    ftq_opts opts{};
    cudaStream_t stream = nullptr;
    int W = 0, M = 0, k = 0;
    int nslot = 0;                // 2 nq_half + 1
    // walker state (complex128 unless noted)
    double2* Y = nullptr;         // FP64 chain: B's since the last QRCP times Q_R [W][M][M]
    double2* Tinv = nullptr;      // T_R^-1                                   [W][M][M]
    double2* G = nullptr;         // G(tau_k), complex128                     [W][M][M]
    double2* work = nullptr;      // LU / QR workspace                        [W][M][M]
    double2* work2 = nullptr;     // triangular-solve workspace (column-major)[W][M][M]
    double2* zbuf[2] = {nullptr, nullptr};   // Horner buffers (FP64) / FP64 bridges (mixed)
    // mixed precision: the chain in FP32 planes split hi + lo for 3xTF32,
    // per walker [hi re | hi im | lo re | lo im], each Kp x LD, zero padded
    int Kp = 0, LD = 0;
    float* Ypl = nullptr;
    float* Yf = nullptr;          // the chain as one FP32 plane (= hi + lo) at the tensor-core tile entries
    float* zpl[2] = {nullptr, nullptr};
    float2* G32 = nullptr;        // G(tau_k) for k < n, complex64            [W][M][M]
    float2* w32 = nullptr;        // FP32 LU workspace                        [W][M][M]
    float2* w2_32 = nullptr;      // FP32 solve workspace = w32 + W M M       [W][M][M]
    bool g64_valid = true;        // G holds the current G(tau) (mixed: only at k = 0, n)
    // TMA descriptors (CUtensorMap, 128 bytes) of the three chain buffers
    alignas(64) unsigned char tmap[3][128] = {};
    const float* tmap_buf[3] = {nullptr, nullptr, nullptr};
    int nct = 1;                  // column tiles of the tensor-core chain (autotuned)
    int64_t wait_limit = -1;      // polls per mbarrier wait of the tensor-core chain (-1: default)
    int qr_nb = 0;                // panel width of the FP32 stabilisation QR (0: widest that fits)
    int green_kind = 0;           // mixed Green kernel: 0 by basis size, 1 tensor cores, 2 CUDA cores
    int4* items = nullptr;        // work list of the tensor-core chain
    int4* items_lr = nullptr;     // the same, compacted by the walkers' ranks (low-rank mixed path)
    int nitems = 0;
    // ragged batch: member systems (owned), CUDA graph of the last propagation
    std::vector<ftq_ctx*> members;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    bool owns_stream = false;
    // a batch member runs on the batch's private stream; calls that read or
    // write caller memory are ordered against the caller's stream
    bool member = false;
    cudaStream_t caller_stream = nullptr;
    double* xbuf = nullptr;       // one slice of internally drawn fields      [W][N_alpha]
    double2* DR = nullptr;        // D_R                                       [W][M]
    double2* phi = nullptr;       // V generator table per walker              [W][nslot]
    float2* phi32 = nullptr;      // the same table in FP32 (mixed path)       [W][nslot]
    double2* hh = nullptr;        // Householder u_0 per column                [W][M]
    double* htau = nullptr;       // Householder tau                           [W][M]
    double* xsum = nullptr;       // Re + Im of the T^-1 update's X (mixed)    [W][M][M]
    // population control: scaled weights, copy counts, parents, copy list [1 + 2W]
    double* pc_w = nullptr;
    int* pc_cnt = nullptr;
    int* pc_parent = nullptr;
    int* pc_pairs = nullptr;
    bool resampled = false;       // a comb happened since the last reset
    // structure factor: per-walker <rho(Q) rho(-Q)>, weights, reduced sums (allocated on first use)
    double2* sq_walker = nullptr;
    double2* sq_w = nullptr;
    double* sq_out = nullptr;
    int* perm = nullptr;          // pivot permutation scratch                 [W][M]
    double* wstate = nullptr;     // [W][WSTRIDE] per-walker state (layout above)
    double* est = nullptr;        // [W][WSTRIDE] per-walker estimators
    double* red = nullptr;        // [16] reduced sums (estimators, mu derivative)
    // time-slice estimates: every track_every-th slice, records {k, E_k, N_k, alive, sum w, scale}
    int track_every = 0;
    int trk_n = 0;
    double* trk = nullptr;        // [n_slices][8]
    double* trk_out = nullptr;    // [n_slices + 1][8] summary read by ftq_slice_estimates
    int* status = nullptr;        // latched numeric status
    size_t bytes = 0;
    std::string err;
    // launch accounting and optional per-launch CUDA-event timing
    int64_t launches[FTQ_K_COUNT] = {};
    bool prof = false;
    struct Span { cudaEvent_t a, b; int kind; };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[FTQ_K_COUNT] = {};
    int64_t prof_n[FTQ_K_COUNT] = {};
};

namespace ftq {

inline cudaEvent_t pool_event(ftq_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one kernel launch: counts it, and when profiling is on records a
// CUDA event pair on the context's stream around it.
struct LaunchScope {
    ftq_ctx* c;
    int kind;
    cudaEvent_t a = nullptr;
    LaunchScope(ftq_ctx* c_, int k) : c(c_), kind(k) {
        c->launches[k] += 1;
        if (c->prof) {
            a = pool_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~LaunchScope() {
        if (c->prof && a) {
            cudaEvent_t b = pool_event(c);
            cudaEventRecord(b, c->stream);
            c->spans.push_back({a, b, kind});
        }
    }
};

// Kernel launchers (fp64_kernels.cu).  All asynchronous on ctx->stream.
cudaError_t launch_init_walkers(ftq_ctx* c);
cudaError_t launch_force_bias(ftq_ctx* c, const double* x);
cudaError_t launch_population_control(ftq_ctx* c, double xi, int* parent_out);
cudaError_t launch_pair_branch(ftq_ctx* c, const double* draws_host, int* parent_out);
cudaError_t launch_structure_factor(ftq_ctx* c, double* per_walker_out);
cudaError_t launch_philox_fields(double* out, uint64_t seed, uint32_t sys, int k0, int n, int W, int na,
                                 cudaStream_t st);
cudaError_t launch_chain(ftq_ctx* c);
cudaError_t launch_qrcp(ftq_ctx* c);
cudaError_t launch_green(ftq_ctx* c, int k, bool update_weights);
cudaError_t launch_estimators(ftq_ctx* c, double* per_walker);
// Estimators of slice k into the next slice record (estimators.cu).
cudaError_t launch_slice_estimate(ftq_ctx* c, int k);
cudaError_t launch_slice_summary(ftq_ctx* c, double* out_dev, int rows);
cudaError_t launch_copy_green(ftq_ctx* c, double2* out);
// complex128 factorisations on explicit buffers
cudaError_t launch_qrcp64(ftq_ctx* c, const double2* Yin, double2* Qout);
// physical = true evaluates the physical A(beta) = B_n ... B_1 (no trial block)
// and takes the overlap ratio without a Gaussian factor (the last step of the
// modified overlap, Eq. ztfix).
cudaError_t launch_green64(ftq_ctx* c, const double2* Y, int k, bool update_weights, bool physical = false);
// dtau times the power of B_T in the trial block at slice k: n - k for the
// overlap of Eq. ftoratio, n for the modified overlap of Eq. ztfix.
double left_scale(const ftq_ctx* c, int k);
// Low-rank truncation of the complex128 path (lowrank.cu).
cudaError_t launch_qrcp_lr(ftq_ctx* c);
cudaError_t launch_green_lr(ftq_ctx* c, const double2* Y, int k, bool update_weights, bool physical);
cudaError_t launch_force_bias_any(ftq_ctx* c, const double* x, const void* G, bool g32);

// Mixed-precision launchers (mixed_kernels.cu).
cudaError_t mixed_init(ftq_ctx* c);
cudaError_t mixed_chain(ftq_ctx* c);
cudaError_t mixed_qrcp(ftq_ctx* c);
cudaError_t mixed_green(ftq_ctx* c, int k);
cudaError_t mixed_sync_g64(ftq_ctx* c);    // make G (complex128) hold G(tau) now

// d<N>/dmu, d<E>/dmu at tau = beta (mu_grad.cu).
cudaError_t launch_mu_grad(ftq_ctx* c, double* per_walker);

// Blocked FP32 Green's function (green_blocked.cu); used while its shared
// memory fits.
size_t green32b_smem(int M);
cudaError_t launch_green32b(ftq_ctx* c, int k, float2* G = nullptr, double* ws = nullptr);
size_t green_tc_smem(int M, int NT);
size_t green_tc_floats(int M);   // workspace floats per walker of the tensor-core Green kernel
int green_tc_tile(int M);
cudaError_t launch_green_tc(ftq_ctx* c, int k, float2* G = nullptr, double* ws = nullptr);
bool green_uses_tc(const ftq_ctx* c);
cudaError_t green_autotune(ftq_ctx* c, float* ms_tc, float* ms_lu);

// Pre-pivoted stabilisation of the mixed chain (qr_mixed.cu).
cudaError_t launch_qr_prepiv(ftq_ctx* c);
cudaError_t qr_autotune(ftq_ctx* c, int* best_nb, float* best_ms);

// Tensor-core chain (chain_tc.cu).
void tc_plan(int M, int nct, int* R, int* NT);
cudaError_t tc_chain_step_batch(ftq_ctx* b, const float* const* zin, float* const* out, int j, int p);
cudaError_t tc_batch_items(ftq_ctx* b);
cudaError_t tc_autotune(ftq_ctx* c, int* best_nct, float* best_ms);
bool tc_supported(int M);
cudaError_t tc_make_maps(ftq_ctx* c);
cudaError_t tc_items_by_rank(ftq_ctx* c);
cudaError_t tc_chain_step(ftq_ctx* c, const float* zin, float* out, const double* zs, const double* os,
                          float alpha);

}  // namespace ftq

/*
 * ftq.h -- C ABI of the GB300 walker-propagation library for phaseless
 * finite-temperature AFQMC (ph-FT-AFQMC) of the 3D uniform electron gas in a
 * plane-wave basis (Lee, Morales, Malone, arXiv:2012.12228).
 *
 * The library owns all walker state in device memory and runs every step of
 * the path in its own sm_103a kernels; there is no CPU fallback.  Calls are
 * ordered on the CUDA stream given in ftq_opts (NULL: the legacy default
 * stream).  Caller buffers are read or written during the call's stream
 * order and never retained.
 *
 * Every function returns FTQ_OK (0) or a negative status; the message of the
 * last failure is available from ftq_last_error().
 *
 * Conventions (fixed, independent of precision):
 *   basis     integer vectors n with |n|^2 <= ncut2 (closed shell with M
 *             members), K = 2 pi n / L, ordered by (|n|^2, nx, ny, nz).
 *   transfers every nonzero n_K' - n_K; the half space is the set whose first
 *             nonzero component is positive, ordered by (|n|^2, nx, ny, nz).
 *             Field alpha = 2q is the A(Q_q) field, alpha = 2q + 1 the B(Q_q)
 *             field, N_alpha = number of all nonzero transfers.
 *   G         complex128 [W][M][M] row-major, G_ij = <c_i c_j^+> for one spin
 *             block (both spin blocks are identical for the unpolarised gas),
 *             the equal-time Green's function at the current imaginary time.
 */
#ifndef FTQ_H
#define FTQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FTQ_OK        0
#define FTQ_EINVAL   -1   /* bad argument or call out of sequence            */
#define FTQ_ECUDA    -2   /* a CUDA runtime call or kernel launch failed      */
#define FTQ_ENUMERIC -3   /* singular pivot or non-finite log-determinant     */
#define FTQ_ETIMEOUT -4   /* a bounded host wait expired                      */
#define FTQ_ENOMEM   -5   /* device allocation failed                         */

/* precision of the slice chain */
#define FTQ_FP64   0      /* every step in complex128                                   */
#define FTQ_MIXED  1      /* B chain in 3xTF32 tensor-core math (tcgen05, FP32 accumulate),
                             FP32 per-slice G and LU, FP64 log-determinant accumulation;
                             stabilisation: FP32 Householder of the pre-pivoted chain,
                             D_R in FP64 and the T^-1 update in double-FP32 (48-bit)
                             arithmetic on the FP32 pipe; complex128 G(beta),
                             estimators and log-weights                                  */
#define FTQ_MIXED_SIMT 2  /* as FTQ_MIXED with the chain on FP32 CUDA cores (measured
                             variant and cross-check of the tensor-core chain)          */
#define FTQ_MIXED_F64UDT 3 /* as FTQ_MIXED with the T^-1 update on the FP64 pipe
                             (measured variant and cross-check of the double-FP32 one)  */

/* weight update */
#define FTQ_PHASELESS 0   /* w <- |I_k| max(0, cos theta_k)  (Eqs. import, phimport, theta) */
#define FTQ_FREE      1   /* w <- w I_k, complex (unconstrained free projection)            */

/* overlap ratio the weight update and the force bias are built on */
#define FTQ_OVERLAP_PAPER    0  /* S_k of Eq. ftoratio: A_k = B_T^(n-k) B_k ... B_1            */
#define FTQ_OVERLAP_MODIFIED 1  /* S~_k of Eq. ztfix: A~_k = B_T^n B_k ... B_1 at every slice;
                                   after slice n the library evaluates G(beta) and
                                   ln det(I + B_n ... B_1) of the physical ensemble and
                                   multiplies each weight by the ratio
                                   r = [det(I + B_n...B_1) / det(I + B_T^n B_n...B_1)]^2,
                                   projected as a slice ratio (|r| max(0, cos arg r) under
                                   FTQ_PHASELESS, r under FTQ_FREE), so the estimators at
                                   tau = beta target the physical ensemble               */

typedef struct ftq_ctx ftq_ctx;

typedef struct {
    int      walkers;          /* W > 0                                                  */
    int      stabilise_every;  /* s: QRCP of the right block every s slices (0 = never)   */
    int      exp_order;        /* p >= 1: Taylor order of exp(V)                          */
    int      precision;        /* FTQ_FP64, FTQ_MIXED, FTQ_MIXED_SIMT or FTQ_MIXED_F64UDT */
    int      constraint;       /* FTQ_PHASELESS or FTQ_FREE                               */
    int      overlap;          /* FTQ_OVERLAP_PAPER or FTQ_OVERLAP_MODIFIED               */
    uint64_t seed;             /* key of the on-device field generator (ftq_fields)       */
    void*    cuda_stream;      /* cudaStream_t the library launches on (NULL = default)  */
    double   force_bias_cap;   /* must be 0 (no cap: the paper applies none); any other
                                  value is rejected with FTQ_EINVAL                       */
    double   low_rank_threshold; /* 0 = full rank.  > 0: low-rank truncation (Sec.
                                    "Exploiting the low-rank structure", Eq. thresh) with
                                    this absolute threshold (the paper uses 1e-6): every
                                    stabilisation keeps the leading columns of the pivoted
                                    QR with |R_jj| >= threshold (at least one), the trial
                                    block keeps its entries >= threshold, and G and
                                    ln det(I + A) come from the Woodbury identity and the
                                    matrix determinant lemma in the kept dimensions.
                                    complex128 path only (FTQ_FP64); FTQ_EINVAL otherwise */
} ftq_opts;

/* One system of a ragged batch (ftq_init_batch). */
typedef struct {
    int    N, M;
    double rs, theta, mu, dtau;   /* as ftq_init_ueg; mu = NaN selects mu_T */
    int    walkers;
    int    reserved;              /* must be 0 */
} ftq_system;

/* Create a UEG system and W walkers at tau = 0 (A(0) = B_T^n).
 *   N      target electron number N-bar (even, 0 < N < 2M)
 *   M      plane-wave basis size; must be a closed-shell count (7, 19, 27, 33, 57, ...),
 *          at most 2047 with FTQ_FP64 and 1021 with the mixed precisions
 *   rs     Wigner-Seitz radius;  L = (4 pi N / 3)^(1/3) rs     (Computational Details)
 *   theta  T / T_F with k_B T_F = (9 pi / 4)^(2/3) / (2 rs^2)  (Eq. fermiT)
 *   mu     chemical potential of B; NaN selects mu = mu_T      (Sec. Phaseless approximation)
 *   dtau   requested time step; n = round(beta / dtau) slices and dtau := beta / n
 * The free-electron trial B_T = exp(-dtau (|K|^2/2 - mu_T)) uses mu_T tuned so
 * that 2 sum_K f_FD = N (Sec. Results, FE trial; Computational Details).
 * Allocates the device walker state (library-owned, freed by ftq_destroy).
 * Errors: FTQ_EINVAL (bad parameters), FTQ_ENOMEM, FTQ_ECUDA. */
int ftq_init_ueg(ftq_ctx** out, int N, int M, double rs, double theta, double mu,
                 double dtau, const ftq_opts* opts);

/* The library's own N(0,1) auxiliary fields (used by ftq_propagate_slices
 * when fields_dev is NULL): Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
 * with counter (alpha / 2, slice index k (0-based), walker, 0) and key = the
 * two 32-bit halves (low, high) of opts.seed; the four output words give
 * u1 = ((w1 << 32 | w0) >> 11 + 1/2) 2^-53 and u2 from (w3, w2) likewise, and
 * the Box-Muller pair x_alpha = sqrt(-2 ln u1) cos(2 pi u2), x_{alpha+1} =
 * sqrt(-2 ln u1) sin(2 pi u2) in FP64 (the paper draws x ~ N(0, 1), Sec.
 * Theory; the generator is this library's choice).
 *   first_slice, n_slices  window [first_slice, first_slice + n_slices) of [0, n)
 *   out_dev     caller-owned device float64 [n_slices][W][N_alpha]
 * FTQ_EINVAL on a window outside [0, n).  Asynchronous on the context stream. */
int ftq_fields(ftq_ctx* ctx, int first_slice, int n_slices, double* out_dev);

/* Density correlations for the static structure factor
 * S(Q) = <rho(Q) rho(-Q)> / N (Results, structure factor) at the current tau,
 * from P = I - G^T by Wick's theorem: per walker
 * <rho(Q) rho(-Q)> = Gamma_Q - Lambda_Q + D_Q with Gamma_Q = (2 rho_Q)(2 rho_-Q),
 * Lambda_Q the exchange sum of the energy estimator and
 * D_Q = 2 sum_{K: K, K+Q in basis} P_{K+Q,K+Q}; and the weighted sums over walkers.
 * Q runs over the 2 N_alpha/2 = N_alpha transfers in slot order: index
 * 2 q is +q and 2 q + 1 is -q for the half-space transfer q of ftq_transfers().
 *   out_host        host, 4 + 2 N_alpha doubles: {Re sum w, Im sum w, s, n_alive,
 *                   then Re, Im of sum w <rho(Q) rho(-Q)> for every Q}, every w
 *                   scaled by exp(-s), s = max ln|w_i| over live walkers
 *   per_walker_dev  nullable device complex128 [W][N_alpha]: <rho(Q) rho(-Q)>
 * Allocates its work buffers (W x N_alpha complex128) on the first call.
 * Synchronises the stream. */
int ftq_structure_factor(ftq_ctx* ctx, double* out_host, void* per_walker_dev);

/* Comb population control between slices (Computational Details: the comb
 * method).  With the phaseless weights w_i = exp(ln|w_i| - max ln|w|) of the
 * alive walkers (dead walkers weigh 0) and their running sums C_i in index
 * order (FP64), W teeth t_k = (k + xi) (S / W), S = C_{W-1}, are placed; walker
 * i receives the teeth in [C_{i-1}, C_i) (the last walker the rest), i.e. n_i
 * copies.  Walkers with n_i >= 1 keep their slot; their extra copies fill the
 * slots of walkers with n_i = 0 (sources and slots each in ascending order),
 * by copying the whole walker state (chain, T^-1, D_R, G, ln det, weight
 * record).  Afterwards every walker is alive with ln|w| = ln(S / W) + max and
 * phase 0.
 *   xi          the comb's uniform draw in [0, 1), supplied by the caller
 *   parent_dev  nullable device int32 [W]: the walker each slot was copied from
 *               (itself for survivors)
 * FTQ_EINVAL for xi outside [0, 1), free-projection contexts, batch handles
 * (comb each member) and W > 65535.  A comb with no walker alive changes
 * nothing and latches FTQ_ENUMERIC.  After a comb, ftq_mu_grad is refused
 * until ftq_reset (the derivative at fixed draws does not extend across the
 * resampling).  Asynchronous on the context stream. */
int ftq_population_control(ftq_ctx* ctx, double xi, int* parent_dev);

/* Pair-branching population control between slices (Computational Details:
 * the method used below Theta = 0.25).  With the weights normalised to their
 * mean, u_i = w_i / (S / W) (w_i as for the comb, S summed in index order),
 * the heavy walkers (u > 2, by decreasing u, ties to the lower index) are
 * paired in turn with the light ones (u < 1/2, by increasing u, ties to the
 * lower index).  Pair k = (a heavy, b light) keeps a when draws[k] <
 * u_a / (u_a + u_b), else b; the kept walker carries (w_a + w_b) / 2 and its
 * whole state is copied into the other slot.  Unpaired walkers are unchanged;
 * the total weight is conserved.
 *   draws_host  host float64 [W / 2], uniform draws in [0, 1), one per pair
 *   parent_dev  nullable device int32 [W]: the walker each slot was copied from
 * FTQ_EINVAL for draws outside [0, 1), free-projection contexts, batch handles
 * and W > 8192.  ftq_mu_grad is refused afterwards until ftq_reset.
 * Synchronises the stream (the draws are read before the call returns). */
int ftq_pair_branch(ftq_ctx* ctx, const double* draws_host, int* parent_dev);

/* Return every walker to tau = 0 (k = 0, unit weights, all alive). */
int ftq_reset(ftq_ctx* ctx);

/* Propagate all walkers over the next n_slices imaginary-time slices
 * (Eqs. B, Abrenda, ftoratio, import, phimport; Sec. Numerical Stabilization).
 * Per slice k: force bias from P(tau_{k-1}) (the optimal force bias), shifted
 * fields y = x - xbar, B_k = e^{-dtau K/2} e^{V(y)} e^{-dtau K/2} applied to the
 * right block, QRCP every s slices, G(tau_k) and ln det(I + A(tau_k)), and the
 * weight update.
 *   fields_dev  device pointer, float64 [n_slices][W][N_alpha] C order, N(0,1)
 *               draws x_k, caller-owned; or NULL: the library draws them
 *               itself, slice by slice, with the generator of ftq_fields().
 * The slice counter may not pass n (FTQ_EINVAL).  Asynchronous: numeric
 * breakdown is latched on the device and reported by ftq_status(). */
int ftq_propagate_slices(ftq_ctx* ctx, int n_slices, const double* fields_dev);

/* Force a QRCP refresh of the right block now (Sec. Numerical Stabilization).
 * A(tau) and G(tau) are unchanged up to rounding. */
int ftq_stabilise(ftq_ctx* ctx);

/* Copy G(tau) of every walker into G_dev (device, complex128 [W][M][M],
 * row-major, caller-owned).  Eq. green; at tau = beta this is (I + A)^-1. */
int ftq_green(ftq_ctx* ctx, void* G_dev);

/* Estimators at the current tau from P = I - G^T (Sec. UEG, local energy):
 * N = 2 tr P, E = E_M + E_1 + E_2 with Gamma_Q and Lambda_Q, per walker, and
 * the weighted sums over walkers (Theory: <O> = sum w O_L / sum w).
 *   out_host        host, 8 doubles: {Re sum w, Im sum w, Re sum wE, Im sum wE,
 *                   Re sum wN, Im sum wN, s, n_alive} where every w is scaled by
 *                   exp(-s), s = max_i ln|w_i| over live walkers.
 *   per_walker_dev  nullable device float64 [W][8]: {ln|w|, arg w, alive,
 *                   Re E, Im E, Re N, Im N, unused}.
 * Synchronises the stream. */
int ftq_estimators(ftq_ctx* ctx, double* out_host, double* per_walker_dev);

/* Derivatives of the estimates with respect to the chemical potential mu of
 * B, at tau = beta, at fixed draws x and with every slice's force bias held at
 * its value on the path (mu tuning: the interacting mu is tuned so that
 * <N> = N-bar, Computational Details).  Every B carries exp(dtau mu), so
 * d ln det(I + A_k)/dmu = k dtau (M - tr G(tau_k)) is accumulated during
 * propagation into d ln|w|/dmu (phaseless: Re d ln S_k - tan(theta_k)
 * Im d ln S_k); at tau = beta dG/dmu = -beta (I - G) G and
 * d<O>/dmu = <dO + O d ln w> - <O><d ln w>.
 *   out_host        host, 8 doubles: {Re d<N>/dmu, Re d<E>/dmu, Re <N>, Re <E>,
 *                   n_alive, s, Im d<N>/dmu, Im d<E>/dmu}
 *   per_walker_dev  nullable device float64 [W][8]: {d ln|w|/dmu, d arg w/dmu,
 *                   Re dE/dmu, Im dE/dmu, Re dN/dmu, Im dN/dmu, 0, 0}
 * FTQ_EINVAL unless the walkers are at tau = beta.  Synchronises the stream. */
int ftq_mu_grad(ftq_ctx* ctx, double* out_host, double* per_walker_dev);

/* Per-walker weights and determinants: device float64 [W][8]
 * {ln|w|, arg w, alive, Re ln det(I+A), Im ln det(I+A), Re gauss_k,
 *  Im gauss_k, unused} where gauss_k = x_k.xbar_k - xbar_k.xbar_k / 2 of the
 * last slice (Eq. import). */
int ftq_weights(ftq_ctx* ctx, double* out_dev);

/* Rank m of every walker's right block (Sec. "Exploiting the low-rank
 * structure": the number of kept scales after the last stabilisation; M on
 * the full-rank path).  ranks_host: caller-owned host int[W]; synchronises the
 * stream. */
int ftq_ranks(ftq_ctx* ctx, int* ranks_host);

/* Read and clear the latched device status: FTQ_OK, FTQ_ENUMERIC (zero or
 * NaN pivot, non-finite log-determinant) or FTQ_ETIMEOUT (a tensor-core
 * kernel gave up a bounded wait on its own copies and left its output
 * unwritten); synchronises the stream. */
int ftq_status(ftq_ctx* ctx, int* status_host);

/* Choose the mixed path's kernel for G(tau_k), k < n (no counterpart in the
 * paper, which computes G by one factorisation per slice): 0 by basis size
 * (tensor cores from M = 384 up), 1 the tensor-core Gauss-Jordan kernel,
 * 2 the CUDA-core blocked LU.  Both compute the same G, ln det and weights to
 * FP32 accuracy; ftq_autotune sets the faster one.  No effect for FP64
 * precision, FTQ_MIXED_SIMT (always the LU) or low rank.
 * Errors: FTQ_EINVAL (NULL context or kind outside 0..2). */
int ftq_set_green_kernel(ftq_ctx* ctx, int kind);

/* Test hook of the failure detection (no counterpart in the paper): every
 * mbarrier wait of the tensor-core kernels (mixed precision: the chain and
 * the Gauss-Jordan G) polls at
 * most `polls` times before it gives up; -1 restores the default of 2^24
 * polls.  A wait that gives up latches FTQ_ETIMEOUT (read by ftq_status), the
 * kernel skips its remaining work, drains its own copies and MMAs with the
 * default bound and frees its tensor memory, so the context stays usable: the
 * chain of that launch is not updated, and ftq_reset starts a clean path.
 * For a batch context the value applies to the batched launches.  Setting a
 * small value makes propagation fail; it exists to exercise the timeout path.
 * Errors: FTQ_EINVAL (NULL context or polls < -1). */
int ftq_set_wait_limit(ftq_ctx* ctx, int64_t polls);

/* Time-slice estimates and their average (Results, "Assessing the Phaseless
 * Constraint": "No Average" is the global estimate at tau = beta, "Average"
 * the global estimate averaged over the time slices).  After
 * ftq_track_estimates(ctx, every) with every > 0, each slice k propagated by
 * ftq_propagate_slices with k % every == 0 is followed by the estimators of
 * every walker from G(tau_k) (the complex128 path: complex128 G; the mixed
 * path: the FP32 G of the slice, complex128 at tau = beta) and by the
 * weighted global estimate of slice k, E_k = sum_w w_k E_L / sum_w w_k and
 * N_k likewise (w_k the walkers' weights at slice k, complex in free
 * projection), recorded on the device.  every = 0 stops recording;
 * ftq_reset clears the record.  Not for batch contexts.
 * Errors: FTQ_EINVAL (every < 0, a batch context), FTQ_ENOMEM. */
int ftq_track_estimates(ftq_ctx* ctx, int every);

/* Read the recorded slice estimates; synchronises the stream.
 *   out_host  host float64 [1 + capacity][8].  Row 0: {n recorded, Re E_avg,
 *             Im E_avg, Re N_avg, Im N_avg, 0, 0, 0}, the averages over the
 *             recorded slices of E_k and N_k (each slice counts once).  Row r
 *             (1 <= r <= min(n, capacity)): {k, Re E_k, Im E_k, Re N_k, Im N_k,
 *             alive walkers, Re of the sum of the scaled weights, ln of the
 *             scale} for the r-th recorded slice.
 * Errors: FTQ_EINVAL (NULL buffer, capacity < 0, tracking never enabled),
 * FTQ_ECUDA. */
int ftq_slice_estimates(ftq_ctx* ctx, double* out_host, int capacity);

/* Integer properties. */
#define FTQ_Q_M          0
#define FTQ_Q_N_ALPHA    1
#define FTQ_Q_N_SLICES   2
#define FTQ_Q_SLICE      3   /* slices propagated since the last reset */
#define FTQ_Q_WALKERS    4
#define FTQ_Q_NCUT2      5
#define FTQ_Q_PRECISION  6
#define FTQ_Q_DEVICE_BYTES 7 /* device bytes owned by the context */
#define FTQ_Q_QR_PANEL   8   /* panel width of the mixed path's FP32 QR (0: default) */
#define FTQ_Q_GREEN_KERNEL 9 /* mixed path's G(tau) kernel for k < n: 1 tensor-core
                                Gauss-Jordan, 2 CUDA-core blocked LU, 0 none (FP64
                                precision or low rank) */
int ftq_query(const ftq_ctx* ctx, int key, int64_t* value);

/* Floating-point properties. */
#define FTQ_F_BETA   0
#define FTQ_F_DTAU   1
#define FTQ_F_MU     2
#define FTQ_F_MU_T   3
#define FTQ_F_L      4
#define FTQ_F_E_M    5   /* E_M = N-bar * (-2.837297 / L) / 2 (Sec. UEG, Madelung term) */
int ftq_query_f64(const ftq_ctx* ctx, int key, double* value);

/* Host copies of the conventions: basis integer vectors [M][3] and
 * half-space transfers [N_alpha/2][3] (int32, host buffers, caller-owned). */
int ftq_basis(const ftq_ctx* ctx, int32_t* nvec_host);
int ftq_transfers(const ftq_ctx* ctx, int32_t* q_host);

/* Ragged batch: nsys (1..8) UEG systems of different basis size propagated
 * together with the mixed-precision path (opts->precision must be FTQ_MIXED;
 * opts->walkers is ignored, each system gives its own).  Every Horner step of
 * the tensor-core chain runs as one persistent launch over the work items
 * (system, walker, 64-row block, column tile) of all systems, and every
 * ftq_batch_propagate call is captured into a CUDA graph that is updated and
 * replayed as one launch.  The batch runs on its own stream, ordered after
 * opts->cuda_stream on entry and before it on exit of every call.  The
 * member systems are ordinary contexts (ftq_batch_member) for ftq_green,
 * ftq_estimators, ftq_weights and ftq_mu_grad; they are destroyed with the
 * batch.  A member keeps running on the batch's stream: every call on it that
 * reads or writes caller device memory first waits for opts->cuda_stream and
 * then makes opts->cuda_stream wait for its own work, so buffers of the
 * caller's stream are safe to use around it.  Not a construct of the paper: it batches independent instances of
 * its slice path (Sec. Computational Details: many independent simulations). */
int ftq_init_batch(ftq_ctx** out, int nsys, const ftq_system* systems, const ftq_opts* opts);
int ftq_batch_member(ftq_ctx* batch, int index, ftq_ctx** member);
/* fields_dev: host array of nsys device pointers, member s float64
 * [n_slices][W_s][N_alpha_s]; every member must stay within its own path. */
int ftq_batch_propagate(ftq_ctx* batch, int n_slices, const double* const* fields_dev);

/* Time the candidate column tilings (1, 2 or 3 column tiles per 64-row
 * block) of the tensor-core chain on the context's own shapes and keep the
 * fastest, likewise the panel width (32, 16 or 8 columns) of the FP32
 * Householder QR of the stabilisation and the kernel of G(tau) (tensor-core
 * Gauss-Jordan or CUDA-core blocked LU, FTQ_Q_GREEN_KERNEL); for a batch
 * every member is tuned.
 * choice / ms: nullable host arrays (one entry per system) receiving the
 * chosen tile count and its time per Horner step.  Uses the scratch buffers
 * of the chain, of the stabilisation and of the estimators; walker state,
 * G(tau) and the status word are not changed. */
int ftq_autotune(ftq_ctx* ctx, int* choice, float* ms);

/* Kernel classes for launch accounting and timing. */
#define FTQ_K_FORCE_BIAS 0   /* force bias + shifted fields + V generator table   */
#define FTQ_K_CHAIN      1   /* one Taylor-Horner step of exp(V) on the chain       */
#define FTQ_K_QRCP       2   /* QRCP stabilisation (mixed: pre-pivoted FP32 QR)      */
#define FTQ_K_GREEN      3   /* G(tau), ln det(I + A) and the weight update         */
#define FTQ_K_ESTIMATORS 4   /* per-walker estimators and the walker reduction      */
#define FTQ_K_INIT       5   /* walker initialisation / reset                      */
#define FTQ_K_BRIDGE     6   /* layout conversions between the FP32 chain and FP64  */
#define FTQ_K_BORDER     7   /* chain entries outside the tensor-core tile         */
#define FTQ_K_FIELDS     8   /* on-device auxiliary-field generator                */
#define FTQ_K_POPULATION 9   /* comb population control                            */
#define FTQ_K_TINV       10  /* mixed path: FP64 update of D_R and T^-1 after the QR */
#define FTQ_K_COUNT      11

/* Start (enable != 0) or stop per-launch timing.  While on, every kernel
 * launch is bracketed by a CUDA event pair on the context's stream; enabling
 * clears the accumulated times.  Timing adds event records between launches
 * and is meant for measurement runs only. */
int ftq_profile(ftq_ctx* ctx, int enable);

/* Synchronise the stream and return, per kernel class, the summed event time
 * in milliseconds of the launches timed since profiling was enabled, and the
 * number of launches made since the context was created (timed or not).
 * Both arrays are host buffers of FTQ_K_COUNT entries; either may be NULL. */
int ftq_profile_read(ftq_ctx* ctx, double* ms_host, int64_t* launches_host);

/* Estimators without any device allocation (the paper has no counterpart;
 * this is a service for callers that cannot let a library allocate device
 * memory: applications whose device memory is owned by a framework pool
 * with a fixed budget, and latency-sensitive loops that must not trigger the
 * implicit device-wide synchronisation of cudaMalloc / cudaFree).
 *
 * Computes, for every walker w, the same per-walker values as
 * ftq_estimators: N = 2 tr P and E = E_M + E_1 + E_2 from P = I - G_w^T for
 * the UEG with N-bar = N electrons, M plane waves and Wigner-Seitz radius rs
 * (the estimators do not depend on Theta, dtau or mu).
 *   G_dev           device, complex128 [W][M][M] row-major (as ftq_green writes)
 *   per_walker_dev  device float64 [W][8]: {0, 0, 1, Re E, Im E, Re N, Im N, 0}
 *   cuda_stream     cudaStream_t to run on (NULL = legacy default stream)
 * Working memory: the momentum-transfer tables are packed into one 4 MiB
 * file-scope device array that every GPU which loads the library keeps until
 * the process exits; bases whose tables do not fit (M above roughly 600)
 * are rejected with FTQ_EINVAL and a message naming the size.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 * The first call on a device looks up the array's device address once
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call rewrites the table region it uses
 * and nothing in the array needs to start at zero.  All calls share the one
 * array: calls that can overlap on the GPU (different streams, or different
 * host threads on the same device) race and must be serialised by the
 * caller.  Each call copies the tables from pageable host memory, so it
 * waits on the host until earlier work on cuda_stream is done before the
 * copy starts; the kernel then runs asynchronously on cuda_stream.  Errors
 * via ftq_last_error(NULL). */
int ftq_estimators_noalloc(int N, int M, double rs, const void* G_dev, int W,
                           double* per_walker_dev, void* cuda_stream);

/* Message of the last failure on ctx (or of the last failed ftq_init_ueg
 * when ctx is NULL).  Never NULL. */
const char* ftq_last_error(const ftq_ctx* ctx);

/* Free the context and its device memory.  NULL is accepted. */
void ftq_destroy(ftq_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FTQ_H */

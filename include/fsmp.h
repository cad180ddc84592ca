/*
 * fsmp.h -- C ABI of the GB300 FSMP library (libfsmp.so).
 *
 * FSMP (Wang et al., "The Fast Stochastic Matching Pursuit for Neutrino and Dark Matter
 * Experiments", arXiv 2403.03156) analyses a PMT waveform by sampling photo-electron (PE)
 * sequences z = {t_1..t_N} from p(z | w, lambda0, t0) (Sec. 2.2, Eq. (pz)) with a Gibbs
 * sampler: a Metropolis-Hastings move on the event time t0, then one reversible-jump move on
 * z (birth / death / update, Sec. 2.4, Eqs. (birth), (death), (update)), each scored by the
 * waveform log-likelihood ratio Delta nu of Appendix A.1 (Eqs. (11)-(18)) computed from a
 * resident Sigma^-1 by Woodbury and determinant-lemma updates.
 *
 * This library runs one chain per waveform on the GPU. Every step of the chain (tables, RNG,
 * proposals, Delta nu, accept/reject, the Sigma^-1 update, summaries) runs in the library's
 * own sm_103a kernels. No function here throws; every function returns an FSMP_* status.
 *
 * Conventions shared by all entry points
 *  - Times are in ns. A waveform's sample s is at t_origin + s * dt_sample_ns. PE times and
 *    t0 live on the grid t_origin + j * grid_ns (R = dt_sample_ns / grid_ns is an integer);
 *    "grid units" below are such j.
 *  - A waveform batch is ragged: waveform i is samples[offsets[i] .. offsets[i+1]).
 *  - The random stream of waveform i is Philox4x64-10 keyed by (seed, wf_id) with
 *    wf_id = wf_ids[i] if given, else index_base + i; the counter is (step, block, 0, 0).
 *    A result therefore depends only on the waveform, its wf_id and the seed: never on the
 *    batch it travels in, its position, the GPU slot it ran in or the other work in flight.
 *  - Pointers named "device" must be device memory of the context's GPU (e.g. from a
 *    PyTorch CUDA tensor); all others are host memory.
 */
#ifndef FSMP_H
#define FSMP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FSMP_OK 0
#define FSMP_ERR_INVALID (-1)   /* bad argument; nothing was queued or launched            */
#define FSMP_ERR_CUDA (-2)      /* a CUDA call failed; the context should be destroyed      */
#define FSMP_ERR_NOMEM (-3)     /* host or device allocation failed / over the memory budget */
#define FSMP_ERR_BUSY (-4)      /* submit queue full; retry after fsmp_poll                  */
#define FSMP_ERR_TIMEOUT (-5)   /* a bounded wait ran out                                   */
#define FSMP_ERR_CLOSED (-6)    /* context is shutting down                                  */

/* ---- per-chain status bits (fsmp_summary.status) ---- */
#define FSMP_ST_CAPACITY 1      /* a birth was refused at N == n_cap (truncated target)      */
#define FSMP_ST_BADDET 2        /* a proposal had det(I + Lambda M) <= 0; it was rejected    */
#define FSMP_ST_DRIFT 4         /* an FP64 refresh found incremental drift above threshold   */
#define FSMP_ST_INVALID 8       /* the waveform's inputs were invalid; the chain did not run */
#define FSMP_ST_NONFINITE 16    /* a non-finite Delta nu was met; the proposal was rejected  */

/* ---- arithmetic of the chain state ---- */
#define FSMP_FP64 0             /* Sigma^-1, s, y and all reductions in FP64                 */
#define FSMP_FP32_REFRESH 1     /* FP32 Sigma^-1 / s / y with compensated reductions; FP64
                                   2x2 algebra, log|Sigma| and log-likelihood; FP64 rebuild of
                                   Sigma^-1, s and log|Sigma| every refresh_every accepts      */

/* ---- kernel form ---- */
#define FSMP_KERNEL_AUTO 0      /* library choice: FSMP_KERNEL_PE                            */
#define FSMP_KERNEL_SMEM 1      /* persistent kernel, one CTA per chain, packed Sigma^-1 in
                                   shared memory                                            */
#define FSMP_KERNEL_GLOBAL 2    /* same kernel with packed Sigma^-1 in global memory (L2/HBM),
                                   for windows too long for shared memory                   */
#define FSMP_KERNEL_PLAIN 3     /* baseline: one launch per chain, full n x n FP64 Sigma^-1 in
                                   global memory                                            */
#define FSMP_KERNEL_PE 4        /* persistent kernel, a warp (or half warp) per chain, state in PE space:
                                   the N x N inverse of C = (sigma_eps^2/sigma_q^2) I + A^T A
                                   (Woodbury on all of A), O(N^2) per accepted move          */

typedef struct fsmp_ctx fsmp_ctx;

#define FSMP_MAX_MIX 8          /* components of the MCP charge mixture                      */

/* Model and engine parameters, copied at fsmp_create. Model terms follow the paper:
 *  - SER (Sec. 3): ser_kind 0 is the ex-Gaussian shifted by 4 sigma,
 *    V(t) = (1/2tau) exp((s^2 - 2(t-4s)tau)/2tau^2) erfc((s^2 - (t-4s)tau)/(sqrt2 s tau)),
 *    normalised to peak 1 on the PE grid; ser_kind 1 subtracts ser_under_frac times a
 *    peak-normalised ex-Gaussian(ser_under_sigma, ser_under_tau) started at the main peak.
 *    The SER is truncated after the last grid point with |V| >= ser_eps, rounded up to whole
 *    samples (L_V samples).
 *  - phi (PE time density about t0, Eq. (pzmu)): phi_kind 0 ex-Gaussian(phi_p1 = sigma,
 *    phi_p2 = tau) with Gaussian mean 0; phi_kind 1 the LS profile of Sec. 3
 *    (tau1 = phi_p1, tau2 = phi_p2). phi := 0 for |t| > phi_support_ns.
 *  - charges N(mu_q, sigma_q^2) marginalised (Sec. 2.1, Appendix A.1); white noise
 *    sigma_noise (Sec. 1).
 *  - MCP charge model (Eq. (mcp-multi-norm), Sec. 2.1; Eq. (mcp), Sec. 2.4; Appendix A.2):
 *    n_mix > 0 Gaussian components, a PE of component e has charge N(mix_mu[e],
 *    mix_sigma[e]^2) with prior probability mix_G[e] (the G(e) must sum to 1); a PE is then
 *    (t, e), e+ ~ G is drawn for every birth and update, and mu_q, sigma_q are unused.
 *    n_mix = 0 is the dynode model. Only FSMP_KERNEL_PE (and AUTO) runs a mixture.
 *  - t0 prior uniform on [t0_lo, t0_hi] (Eq. (t0prior)); sample_t0 = 0 holds t0 fixed.
 *  - jump probabilities J, J, 1 - 2J (Sec. 2.4); n_cap = PE capacity per chain. */
typedef struct {
  double dt_sample_ns, grid_ns;
  int ser_kind;
  double ser_sigma, ser_tau, ser_under_frac, ser_under_sigma, ser_under_tau, ser_eps;
  int phi_kind;
  double phi_p1, phi_p2, phi_support_ns;
  double mu_q, sigma_q, sigma_noise;
  double t0_lo, t0_hi;
  int sample_t0;
  double jump_J;
  int n_cap;
  int n_max;               /* longest window (samples) any batch may carry                   */
  int precision;           /* FSMP_FP64 | FSMP_FP32_REFRESH                                  */
  int refresh_every;       /* K accepted moves between FP64 refreshes (FP32 mode)            */
  double drift_tol;        /* relative refresh drift that sets FSMP_ST_DRIFT (0: 5e-2)       */
  int kernel;              /* FSMP_KERNEL_*                                                  */
  int threads_per_chain;   /* CTA size: 0 = autotuned, else 32..512, a multiple of 32; with
                              FSMP_KERNEL_PE each warp of the CTA runs its own chain        */
  size_t device_mem_budget;/* bytes the serving loop may hold for admitted requests (0: 4 GiB) */
  int device;              /* CUDA device ordinal                                            */
  int max_queued;          /* submit queue depth before FSMP_ERR_BUSY (0: 1024)              */
  int n_streams;           /* concurrent launch streams of the serving loop (0: 4)           */
  int pe_tile;             /* FSMP_KERNEL_PE: PEs per chain whose C^-1 stays in shared memory
                              (0: autotuned); a chain moves C^-1 to global memory beyond it */
  int pe_ctas_per_sm;      /* FSMP_KERNEL_PE: resident CTAs per SM (0: as many as fit); fewer
                              keep the chains' global C^-1 slots in L2 when chains are large  */
  int pe_lanes;            /* FSMP_KERNEL_PE: lanes per chain, 32 (a warp) or 16 (two chains per
                              warp; n_cap <= 192 only); 0: 32 until fsmp_autotune picks one.
                              The lane count sets the order of the chain's sums, so results
                              for another count agree up to rounding, not bit for bit       */
  int n_mix;               /* MCP charge mixture: number of components (0: dynode model)     */
  double mix_G[FSMP_MAX_MIX], mix_mu[FSMP_MAX_MIX], mix_sigma[FSMP_MAX_MIX];
} fsmp_params;

/* One waveform's posterior summaries (after burn_in steps). t0 is in absolute ns.
 * mean_Q is the posterior-mean total charge, N mu_q + sigma_q^2 u^T Sigma^-1 y with
 * u = sum_k a_k (the Gaussian posterior of the marginalised charges of Eq. (mgauss)).
 * logL = log p(w | z_final) (Appendix A.1), logdet = log|Sigma(z_final)|.
 * drift_max: FP32 mode, the largest relative difference between the incrementally updated
 * state and its FP64 rebuild seen at a refresh (n_refresh of them).
 * alg_bytes: bytes of chain state the method had to move (per proposal the U x U lower
 * triangle of Sigma^-1 and s on U; per accepted jump Sigma^-1 a, the packed rank-2 update
 * read and write, and s), for roofline accounting.
 * acc / prop count accepted / proposed birth, death, update moves (an update by zero grid
 * steps is proposed but not counted as accepted). */
typedef struct {
  double mean_N, var_N, mean_t0, var_t0, mean_Q, var_Q, logL, logdet;
  double drift_max, alg_bytes;
  double lambda_hat;             /* lambda_FSMP = argmax_lambda -lambda + log sum_N h_N
                                    (lambda / lambda0)^N over the chain's N samples h
                                    (Eq. (reduce-mu0)); 0 if every sample has N = 0 */
  /* Mean and variance over the samples of the Wasserstein scalars of the PE sequence, the
   * convergence representatives of Sec. 3.2: a dummy PE at t = 0, e = 0 joins the sequence
   * (so that an empty z is a distribution too) and the scalar is the 1-Wasserstein distance
   * from the sequence to the dummy alone, sum_k |t_k| / (N + 1) for the PE times (ns from the
   * window's first sample) and sum_k e_k / (N + 1) for the MCP components (0 for the dynode
   * model). */
  double mean_wt, var_wt, mean_we, var_we;
  int32_t acc[3], prop[3];
  int32_t acc_t0, prop_t0, N_final, k0_final, status, n_samples, n_refresh, reserved;
} fsmp_summary;

/* One chain step (testing aid): log acceptance ratios of the t0 move (la0) and of the jump
 * (la), the log uniforms they were compared with, Delta nu, N and the t0 grid index after
 * the step, the jump type (0 birth, 1 death, 2 update) and flags (1 t0 proposed, 2 t0
 * accepted, 4 jump accepted, 8 jump was a no-op update). -inf marks a forced reject, NaN a
 * move that was not made. */
typedef struct {
  double la0, lu0, la, lu, dnu;
  int32_t N, k0, jump, flags;
} fsmp_trace;

/* Host batch for fsmp_submit. All arrays are host memory and are copied during the call;
 * the caller may free them once fsmp_submit returns. Optional arrays may be NULL:
 * T_lo / T_hi (PE solution space in grid units, default the whole window [0, n R)),
 * t0_init (ns, default the grid point nearest the middle of the t0 prior), wf_ids. */
typedef struct {
  uint64_t request_id, seed, index_base;
  int n_waveforms, n_steps, burn_in, record_trace;
  const float* samples;
  const int32_t* offsets;        /* n_waveforms + 1 entries, offsets[0] == 0 */
  const double* lambda0;         /* Poisson expectation guess per waveform, Sec. 2.2 */
  const double* t_origin_ns;     /* time of sample 0 per waveform (NULL: 0)           */
  const int32_t* T_lo;
  const int32_t* T_hi;
  const double* t0_init;
  const uint64_t* wf_ids;
} fsmp_batch;

/* A finished request. Arrays are owned by the library and stay valid until the next
 * fsmp_poll or fsmp_destroy. latency_s = completion time - submit time (host clock). */
typedef struct {
  uint64_t request_id;
  int n_waveforms, status;       /* status: FSMP_OK or the error that ended the request */
  const fsmp_summary* summaries; /* n_waveforms entries                                  */
  const fsmp_trace* trace;       /* n_waveforms * n_steps entries, or NULL               */
  double latency_s;
} fsmp_result;

/* Device-resident batch for fsmp_run_device: every pointer is device memory. n_max_hint
 * bounds the longest window in the batch (0: params.n_max); windows above it are flagged
 * FSMP_ST_INVALID. out receives n_waveforms summaries; trace (may be NULL) receives
 * n_waveforms * n_steps records. */
typedef struct {
  int n_waveforms, n_steps, burn_in, n_max_hint;
  uint64_t seed, index_base;
  const float* samples;
  const int32_t* offsets;
  const double* lambda0;
  const double* t_origin_ns;     /* may be NULL */
  const int32_t* T_lo;           /* may be NULL */
  const int32_t* T_hi;           /* may be NULL */
  const double* t0_init;         /* may be NULL */
  const uint64_t* wf_ids;        /* may be NULL */
  fsmp_summary* out;
  fsmp_trace* trace;             /* may be NULL */
  /* Initial state (may be NULL; FSMP_KERNEL_PE only): waveform i starts from the PEs
   * z_init[i * z_stride + k], k < min(n_init[i], z_stride) (grid indices, as LucyDDM gives
   * them, Sec. 2.3) instead of an empty z. More than n_cap PEs are cut to n_cap and flagged
   * FSMP_ST_CAPACITY. With the MCP mixture each starts as the most probable component. */
  const int32_t* z_init;
  const int32_t* n_init;
  int z_stride;
  /* PE-time histogram (may be NULL; FSMP_KERNEL_PE only): after burn-in, every step adds one
   * to pe_hist[i * pe_hist_width + (j - T_lo)] for each PE of waveform i at grid index j with
   * T_lo <= j < T_lo + pe_hist_width (T_lo = 0 without a T_lo array); divided by n_samples
   * it is the posterior mean PE count per grid point. The caller zeroes it. */
  uint32_t* pe_hist;
  int pe_hist_width;
} fsmp_device_batch;

/* LucyDDM (Sec. 2.3): Lucy's iterative deconvolution of each waveform of a device batch by
 * the SER at the sample times, v(m) = V(m dt) / S (m < L_V, S = sum_m V(m dt)), of the data
 * d(t) = max(w(t), 0) / S, from a uniform start with the sum of d, for n_iter iterations
 * (FP32). The taus with q-hat(tau) > thresh give the initial PEs at grid indices tau R, the
 * solution space T = [t_min - 4 ns, t_max + 4 ns] on the PE grid, and t0 = t_origin + t_min --
 * the inputs T_lo, T_hi, t0_init, z_init, n_init of a fsmp_device_batch. A waveform with no
 * such tau gets n_init = 0, T = [0, n R) and t0_init = NaN (the paper leaves it out). Every
 * pointer is device memory; samples / offsets as in fsmp_device_batch with offsets[0] = 0. */
typedef struct {
  int n_waveforms, n_max_hint;   /* n_max_hint: longest window (0: params.n_max)             */
  const float* samples;
  const int32_t* offsets;
  const double* t_origin_ns;     /* may be NULL (0)                                          */
  int n_iter;                    /* Lucy iterations (the paper: 2000)                        */
  double thresh;                 /* initial-PE threshold on q-hat (the paper: 0.1)           */
  float* q_out;                  /* may be NULL; else q-hat of waveform i, tau = -L_V+1 .. n-1,
                                    at q_out[offsets[i] + i (L_V - 1)]                       */
  int32_t* T_lo;                 /* [n_waveforms]                                            */
  int32_t* T_hi;                 /* [n_waveforms] (exclusive)                                */
  double* t0_init;               /* [n_waveforms]                                            */
  int32_t* z_init;               /* [n_waveforms * z_stride] (may be NULL if z_stride = 0)   */
  int32_t* n_init;               /* [n_waveforms]: taus found (only z_stride are stored)     */
  int z_stride;
  int32_t* status;               /* [n_waveforms]: 0, or FSMP_ST_INVALID (empty or too long)  */
} fsmp_lucy_batch;

/* Run LucyDDM on `stream` (asynchronous). Returns FSMP_OK, FSMP_ERR_INVALID (bad arguments,
 * window longer than params.n_max or than shared memory allows) or FSMP_ERR_CUDA. */
int fsmp_lucyddm(fsmp_ctx* ctx, const fsmp_lucy_batch* batch, void* stream);

/* Library and device facts, and the launch shape chosen for each kernel form. */
typedef struct {
  int device, sm_count, smem_per_block_optin, ser_len, R, L_V;
  int n_smem_max;                /* longest window whose Sigma^-1 fits shared memory      */
  int threads_per_chain, ctas_per_sm;
  size_t scratch_bytes;          /* device scratch the context holds                     */
  char name[64];
  long long n_launches;          /* chain-kernel launches made by this context so far     */
} fsmp_info;

/* Create a context on params->device: validates params, computes the SER and phi tables on
 * the GPU (Sec. 3 formulas), allocates device scratch and starts the serving loop.
 * Returns FSMP_OK, FSMP_ERR_INVALID, FSMP_ERR_CUDA or FSMP_ERR_NOMEM; *out is set only on
 * FSMP_OK and is owned by the caller until fsmp_destroy. */
int fsmp_create(const fsmp_params* params, fsmp_ctx** out);

/* Queue a host batch (copied before returning). Non-blocking: FSMP_ERR_BUSY when the queue
 * holds max_queued requests; FSMP_ERR_INVALID for malformed batches (nothing queued);
 * FSMP_ERR_NOMEM when a single request exceeds the device memory budget. The serving loop
 * admits queued requests as device memory frees, packs them into launches, and overlaps
 * their work on the GPU (continuous batching). */
int fsmp_submit(fsmp_ctx* ctx, const fsmp_batch* batch);

/* Collect up to max finished requests, waiting up to timeout_ms (0: do not wait, < 0: wait
 * forever) for the first one. Returns the number written to out (0 on timeout) or a
 * negative FSMP_ERR_*. */
int fsmp_poll(fsmp_ctx* ctx, fsmp_result* out, int max, int timeout_ms);

/* Drain in-flight work (queued but unstarted requests are cancelled), free everything. */
int fsmp_destroy(fsmp_ctx* ctx);

/* Run a device-resident batch on `stream` (a cudaStream_t; NULL = the legacy default
 * stream). Enqueues kernels only: no host synchronisation, no host<->device copies. The
 * context's device scratch is shared by all calls on the context: calls on different
 * streams must not overlap. Returns FSMP_ERR_INVALID for bad arguments, FSMP_ERR_CUDA if a
 * launch fails. */
int fsmp_run_device(fsmp_ctx* ctx, const fsmp_device_batch* batch, void* stream);

/* Gelman-Rubin potential scale reduction R of one scalar over m >= 2 chains of the same
 * waveform (the convergence check of Sec. 3), from their summaries. With n samples per chain
 * (n_samples, equal for all, n >= 2), chain means x_j and variances v_j of the field
 * (FSMP_RHAT_N: N; FSMP_RHAT_T0: t0; FSMP_RHAT_Q: the charge summary):
 *   W = (1/m) sum_j v_j n / (n - 1),   B / n = (1/(m-1)) sum_j (x_j - mean x)^2,
 *   V = (n - 1) / n W + B / n,          R = sqrt(V / W)
 * (the point estimate of Gelman and Rubin, 1992, without a degrees-of-freedom correction).
 * *rhat = 1 when W = 0 and all means agree, +inf when W = 0 and they do not. Host only.
 * Returns FSMP_OK or FSMP_ERR_INVALID. The paper has no code for it; it quotes R < 1.1. */
#define FSMP_RHAT_N 0
#define FSMP_RHAT_T0 1
#define FSMP_RHAT_Q 2
#define FSMP_RHAT_WT 3          /* the Wasserstein scalar of the PE times {t_i} (Sec. 3.2)     */
#define FSMP_RHAT_WE 4          /* the Wasserstein scalar of the MCP components {e_i}          */
int fsmp_gelman_rubin(const fsmp_summary* chains, int m, int field, double* rhat);

/* The convergence check as Sec. 3.2 plots it: the degrees-of-freedom corrected potential scale
 * reduction of a scalar over m >= 2 chains of the same waveform, with its upper confidence
 * limit (Gelman and Rubin 1992, Sec. 3, with the correction (d + 3) / (d + 1) of Brooks and
 * Gelman 1998). From the chains' summaries (n samples each, n >= 2): chain means x_j and
 * within-chain variances s2_j = v_j n / (n - 1); across chains, with m - 1 denominators,
 * var(x), var(s2), cov(s2, x^2), cov(s2, x) and xx = mean of x_j:
 *   W = mean s2_j, B = n var(x), V = (n - 1) / n W + (1 + 1/m) B / n,
 *   var(V) = [(n - 1)^2 var(s2) / m + (1 + 1/m)^2 2 B^2 / (m - 1)
 *             + 2 (n - 1)(1 + 1/m)(n / m)(cov(s2, x^2) - 2 xx cov(s2, x))] / n^2,
 *   d = 2 V^2 / var(V),  c = (d + 3) / (d + 1)  (1 if var(V) = 0),
 *   rhat  = sqrt(c [(n - 1) / n + (1 + 1/m) (B / W) / n]),
 *   upper = the same with B / W times the F(m - 1, 2 W^2 m / var(s2)) quantile at
 *           (1 + confidence) / 2 (chi2(m - 1) / (m - 1) when var(s2) = 0).
 * The paper plots the 90 % upper limit: confidence = 0.9. W = 0 gives 1 (all means equal) or
 * +inf. Host only. Returns FSMP_OK or FSMP_ERR_INVALID (m < 2, n < 2, unequal n, confidence
 * outside (0, 1), unknown field). */
int fsmp_gelman_diag(const fsmp_summary* chains, int m, int field, double confidence, double* rhat,
                     double* upper);

/* Launch shape of the PE-space kernel chosen by fsmp_autotune. */
typedef struct {
  int pe_tile;                   /* PEs per chain whose C^-1 stays in shared memory          */
  int chains_per_cta;            /* chains per CTA (warps x 32 / lanes_per_chain)            */
  int ctas_per_sm;               /* resident CTAs per SM (0: as many as fit)                 */
  int n_tried;                   /* candidate shapes timed                                   */
  double best_steps_per_s;       /* MCMC steps/s of the chosen shape on the trial            */
  double default_steps_per_s;    /* the same for the shape the context started with          */
  int lanes_per_chain;           /* 32 or 16                                                  */
} fsmp_tune;

/* Autotune the launch shape of the PE-space kernel (FSMP_KERNEL_PE contexts) on a device
 * batch laid out as for fsmp_run_device: time trial runs of its first `sample` waveforms for
 * `trial_steps` MCMC steps in each candidate shape -- lanes per chain (only if the context
 * was created with pe_lanes = 0), shared-memory tile of C^-1, warps per CTA and resident CTAs
 * per SM -- and keep the fastest for the context's later launches. The batch's own output and
 * trace buffers are not touched (the trials write to scratch). Later results do not depend on
 * the tile, warps or CTAs: a chain's arithmetic is the same in each. They do depend, up to
 * rounding, on the lane count; fix pe_lanes for results reproducible bit for bit.
 * Blocks until the trials finish. Call it with no request in flight on the context. Returns
 * FSMP_OK (out, if not NULL, describes the choice), FSMP_ERR_INVALID (not a PE-space context,
 * bad arguments) or FSMP_ERR_CUDA / FSMP_ERR_NOMEM. */
int fsmp_autotune(fsmp_ctx* ctx, const fsmp_device_batch* batch, int sample, int trial_steps, fsmp_tune* out);

/* fsmp_run_device for callers that cannot allocate device memory. The paper has no
 * counterpart: this is an integration aid. Some callers cannot call cudaMalloc -- code that
 * runs under a framework allocator owning all device memory, or in a service that forbids
 * allocation after start-up -- and so cannot create an fsmp_ctx (which allocates its tables
 * and scratch). This entry point takes the parameters directly, allocates nothing, and keeps
 * all device scratch it needs (the model tables and the per-CTA FP64 refresh workspaces of
 * the FP32 chain kernel) in one static 64 MiB device array that every GPU loading this code
 * holds until the process exits. The caller passes inputs and outputs as in fsmp_run_device.
 *  - Only precision FSMP_FP32_REFRESH, the dynode charge model (n_mix = 0), windows of at
 *    most 256 samples, n_cap <= 64, phi_support_ns / grid_ns <= 32768 and SER scans of at
 *    most 16384 grid points; anything else returns FSMP_ERR_INVALID (see fsmp_last_error()).
 *  - The first call on a device sets up that device (it resolves the array's address and the
 *    kernel's shared-memory limit), and the first call with a new set of model parameters
 *    rebuilds the tables and synchronises `stream` once: make such a call before any stream
 *    capture.
 *  - All calls share the array and leave it holding the last call's tables and workspaces.
 *    Calls on one stream run in order and are safe whatever their parameters; calls on
 *    different streams that overlap on the GPU race on it.
 *  - params are checked as fsmp_create checks them (threads_per_chain 0 or a multiple of 32
 *    in 32..512, finite mu_q, ...) before anything is enqueued.
 * The current device is restored on return. Returns FSMP_OK, FSMP_ERR_INVALID or
 * FSMP_ERR_CUDA. */
int fsmp_run_device_noalloc(const fsmp_params* params, const fsmp_device_batch* batch, void* stream);

/* The device-computed tables (testing aid): the peak-normalised SER on the PE grid
 * (ser_out, up to max_ser entries; *ser_len gets its length L_V * R) and phi, log phi on grid
 * offsets d in [d_lo, d_lo + count) (phi_out / logphi_out may be NULL). Synchronous. */
int fsmp_get_tables(fsmp_ctx* ctx, double* ser_out, int max_ser, int* ser_len, int d_lo,
                    int count, double* phi_out, double* logphi_out);

int fsmp_get_info(fsmp_ctx* ctx, fsmp_info* out);

/* Philox4x64-10 blocks computed on the GPU (testing aid): out[4i..4i+4) = Philox(ctrs[4i..],
 * key). ctrs and out are host arrays of 4 * n words. Synchronous. */
int fsmp_philox_blocks(fsmp_ctx* ctx, const uint64_t key[2], const uint64_t* ctrs, int n,
                       uint64_t* out);

/* lambda_FSMP (Eq. (reduce-mu0), Sec. 2.2) of given N histograms, computed on the GPU by the
 * same device function every chain of fsmp_run_device ends with (testing aid): out[i] = the
 * maximiser over lambda >= 0 of -lambda + log sum_N h_i[N] (lambda / lambda0[i])^N, with h_i =
 * hist[i (n_max + 1) .. (i + 1)(n_max + 1)) the counts of N = 0 .. n_max, on `lanes` (32 or 16)
 * lanes per histogram as a chain of that lane count would run it; 0 if only N = 0 was counted,
 * NaN if no N was. hist, lambda0 and out are host arrays of n_hist entries (hist of
 * n_hist (n_max + 1)). Synchronous. Returns FSMP_OK, FSMP_ERR_INVALID, FSMP_ERR_NOMEM or
 * FSMP_ERR_CUDA. */
int fsmp_lambda_mle(fsmp_ctx* ctx, const int32_t* hist, int n_hist, int n_max, const double* lambda0, int lanes,
                    double* out);

/* Roofline denominators measured on the context's GPU (the paper has no counterpart; it is
 * a measurement aid): shared-memory load bandwidth in GB/s (16-byte loads, 4 CTAs per SM),
 * and FP64 / FP32 FMA throughput in TFLOP/s (2 flops per FMA). Synchronous, ~0.1 s. */
int fsmp_measure_peaks(fsmp_ctx* ctx, double* smem_gbs, double* fp64_tflops, double* fp32_tflops);

const char* fsmp_strerror(int status);

/* A description of the last failure of an fsmp_* call made by the calling thread (the
 * failing CUDA call and its error string, or the argument that was rejected); "" if none.
 * The string is owned by the library and valid until the thread's next fsmp_* call. */
const char* fsmp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif

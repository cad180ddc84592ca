/*
 * fsmp_oracle.h -- plain FP64 CPU oracle of the FSMP chain.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this library. The product path (the CUDA
 * library under paper_2403_03156_gb300/) never links, imports or calls it, and this
 * file shares no code, header, table or constant generator with it.
 *
 * Source of every formula: Wang et al., "The Fast Stochastic Matching Pursuit for
 * Neutrino and Dark Matter Experiments" (arXiv 2403.03156):
 *   waveform model            Eq. (waveform), Sec. 1
 *   Poisson-process prior     Eq. (pzmu), Sec. 2.2
 *   Gibbs / MH on t0          Sec. 2.4 (t0 acceptance), Sec. 2.2 (Gibbs framework)
 *   birth / death / update    Eqs. (birth), (death), (update), Sec. 2.4
 *   posterior ratio           Eq. (delta-nu) and the ratio above it, Sec. 2.4
 *   jump probabilities J      Sec. 2.4 (J = 1/4, empty / single-PE rules)
 *   proposal h(t)             Sec. 2.4, last equation
 *   SER and phi               Sec. 3 (SER formula; LS two-exponential phi)
 *   marginal likelihood       Appendix A.1, Eq. (mgauss) and the log-density below it
 *   rank-2 jump, Woodbury     Appendix A.1, Eqs. (11), (12), (14), (DeltaU), (16)-(18)
 *   LucyDDM initial state     Sec. 2.3 (Lucy's iteration, the solution space T, initial z, t0)
 *   MCP charge model          Eq. (mcp-multi-norm) (Sec. 2.1), Eq. (mcp) (Sec. 2.4),
 *                             Eq. (mcp-pzmu) and the redefined U, Sigma, Lambda (Appendix A.2)
 *
 * Readings where the paper is silent (grid, t0 prior, tie rules, RNG layout) are the
 * ones listed in the repository's design notes; each is restated where it is used.
 *
 * Parity pins: every function here is checked in tests/ against something other than
 * itself (scipy / numpy library routines, closed forms, brute-force enumeration of the
 * posterior on tiny grids, prior-only limits, numpy's Philox4x64 generator).
 */
#ifndef FSMP_ORACLE_H
#define FSMP_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_MIX 8

typedef struct {
  double dt_sample_ns;     /* sample period (1 ns in the paper, Sec. 2.3 / Sec. 3)          */
  double grid_ns;          /* PE / t0 time grid; dt_sample_ns / grid_ns must be an integer R */
  int    ser_kind;         /* 0: ex-Gaussian SER of Sec. 3; 1: same plus an undershoot term  */
  double ser_sigma, ser_tau;
  double ser_under_frac, ser_under_sigma, ser_under_tau;
  double ser_eps;          /* SER support: last grid point with |V| >= ser_eps (peak = 1)   */
  int    phi_kind;         /* 0: ex-Gaussian(phi_p1 = sigma, phi_p2 = tau); 1: LS (tau1,tau2) */
  double phi_p1, phi_p2;
  double phi_support_ns;   /* phi(t) := 0 for |t| > phi_support_ns                           */
  double mu_q, sigma_q;    /* dynode charge model N(mu_q, sigma_q^2), Sec. 2.1               */
  double sigma_noise;      /* white noise sigma_epsilon, Sec. 1                              */
  double t0_lo, t0_hi;     /* uniform t0 prior, Eq. (t0prior)                                */
  int    sample_t0;        /* 0: t0 held fixed                                               */
  double jump_J;           /* J of Sec. 2.4 (1/4)                                            */
  int    n_cap;            /* PE capacity: a birth at N == n_cap is rejected                  */
  int    prior_only;       /* test switch: Delta nu := 0 (samples the prior restricted to T) */
  /* MCP charge model (Eq. (mcp-multi-norm)): n_mix Gaussian components, PE of component e has
   * charge N(mix_mu[e], mix_sigma[e]^2) with probability mix_G[e]; n_mix = 0 is the dynode
   * model N(mu_q, sigma_q^2) above */
  int    n_mix;
  double mix_G[ORC_MAX_MIX], mix_mu[ORC_MAX_MIX], mix_sigma[ORC_MAX_MIX];
} orc_params;

/* One record per chain step. la0 / la are log acceptance ratios (-inf = forced reject,
 * NaN = no such move); lu0 / lu are the log uniforms they were compared with. */
typedef struct {
  double la0, lu0, la, lu, dnu;
  int32_t N, k0, jump, flags;
  /* the Wasserstein scalars of the state after the step (orc_pe_wasserstein): of the PE times
   * {t_i} (ns from the window's first sample) and of the MCP components {e_i} */
  double wt, we;
} orc_trace;

enum { ORC_F_T0_PROPOSED = 1, ORC_F_T0_ACCEPTED = 2, ORC_F_ACCEPTED = 4, ORC_F_NOOP = 8,
       ORC_F_T0_DISAGREE = 16, ORC_F_DISAGREE = 32 };
enum { ORC_JUMP_BIRTH = 0, ORC_JUMP_DEATH = 1, ORC_JUMP_UPDATE = 2 };
enum { ORC_ST_CAPACITY = 1, ORC_ST_BADDET = 2, ORC_ST_NONFINITE = 16, ORC_ST_DISAGREE = 32 };
enum { ORC_MODE_DEFINITION = 0, ORC_MODE_INCREMENTAL = 1 };

typedef struct {
  double mean_N, var_N, mean_t0, var_t0, mean_Q, var_Q, logL, logdet;
  int32_t acc[3], prop[3];
  int32_t acc_t0, prop_t0, N_final, k0_final, status, n_samples;
  double lambda_hat;  /* lambda_FSMP of the chain's N samples (Eq. (reduce-mu0)); 0 if none */
  /* mean and population variance over the samples of the Wasserstein scalars of {t_i} and
   * {e_i} (orc_pe_wasserstein; the convergence check of Sec. 3.2) */
  double mean_wt, var_wt, mean_we, var_we;
  /* Words of chain state the method moves, counted from the chain's own path for the roofline's
   * algorithmic bytes (a measurement count, not part of the chain's arithmetic): per scored
   * birth or update N + 2p + 2|S+| + p^2 + p (p = PEs whose samples in the window overlap the new
   * PE's, |S+| its samples in the window), per scored death or update 2 more, per accepted move
   * N p + N'(N' + 1) + 2N' (N' = N after it), plus 2|S-| + N when a PE leaves and 2|S+| when one
   * arrives (|S-| the leaving PE's samples in the window). */
  double alg_words;
} orc_summary;

/* 1-Wasserstein distance between the empirical distributions (equal weights) of a[0..na) and
 * b[0..nb) on the real line: the integral of |F_a(x) - F_b(x)| over x, with F the empirical
 * CDFs (na, nb >= 1). */
double orc_wasserstein1(const double* a, int na, const double* b, int nb);

/* The scalar the convergence check of Sec. 3.2 takes from a trans-dimensional PE sequence:
 * a dummy PE (t = 0, e = 0) joins every sequence, so that an empty z is a distribution too,
 * and the scalar is the 1-Wasserstein distance from the sequence with its dummy to the dummy
 * alone. v[0..N) are the PEs' times in ns from the window's first sample (or their MCP
 * components). */
double orc_pe_wasserstein(const double* v, int N);

/* lambda_FSMP = argmax_lambda l(lambda), l = -lambda + log sum_N h[N] (lambda / lambda0)^N
 * (Eq. (reduce-mu0) with the samples counted by N in h[0 .. n_max]), by a dense grid over
 * [0, 2 max{N : h[N] > 0} + 10] and golden-section refinement around the best grid point. */
double orc_lambda_mle(const double* h, int n_max, double lambda0);

/* Batch description: waveform i is samples[offsets[i] .. offsets[i+1]). Optional arrays may
 * be NULL: T_lo/T_hi (default: whole window [0, n*R)), t0_init (default: prior midpoint). */
typedef struct {
  int n_waveforms;
  const float* samples; const int32_t* offsets;
  const double* lambda0; const double* t_origin_ns;
  const int32_t* T_lo; const int32_t* T_hi; const double* t0_init;
  uint64_t seed, index_base;
  const uint64_t* wf_ids;  /* optional per-waveform RNG index (default index_base + i) */
  int n_steps, burn_in;
  const uint8_t* forced;   /* optional [n_waveforms * n_steps]: bit0 t0 decision, bit1 z decision */
  double* occ;             /* optional [n_waveforms * occ_width]: time-averaged PE count at grid
                              index T_lo + c (c < occ_width) after burn-in (a PE-time histogram) */
  int occ_width;
  double* occ_e;           /* optional [n_waveforms * max(n_mix, 1)]: time-averaged number of PEs
                              of each MCP component after burn-in */
  const int32_t* z_init;   /* optional [n_waveforms * z_stride]: initial PE grid indices (the
                              LucyDDM initial state, Sec. 2.3); NULL starts from an empty z */
  const int32_t* n_init;   /* their counts (required with z_init) */
  int z_stride;
} orc_batch;

/* Philox4x64-10 block function. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* n blocks: out[4i..4i+4) = Philox(ctrs[4i..4i+4), key). */
void orc_philox_blocks(const uint64_t key[2], const uint64_t* ctrs, int n, uint64_t* out);
/* The 8 uniforms of one chain step (two Philox blocks), in (0,1). */
void orc_step_uniforms(uint64_t seed, uint64_t wf_index, uint64_t step, double u[8]);
/* The uniform that draws the MCP component of a born or updated PE (n_mix > 1): the first
 * output of a third block, counter (step, 2, 0, 0). */
double orc_step_uniform_e(uint64_t seed, uint64_t wf_index, uint64_t step);

/* SER V_PE(t) (Sec. 3 formula, not normalised) and phi(t). */
double orc_ser_raw(const orc_params* p, double t_ns);
double orc_phi(const orc_params* p, double t_ns);
/* Peak-normalised SER table on the PE grid. Returns the table length Lt = L_V * R, or a
 * negative error. Fills up to max_len entries of out; *peak_out gets the normaliser. */
int orc_ser_table(const orc_params* p, double* out, int max_len, double* peak_out);

/* log p(w | z) by building Sigma(z), U(z) and a Cholesky factorisation (Appendix A.1). */
double orc_logp_definition(const orc_params* p, const float* w, int n, const int32_t* j, int N,
                           double* logdet_out, double* quad_out);
/* The same for z = {(t_k, e_k)} of the MCP model (Appendix A.2); e may be NULL (all 0). */
double orc_logp_definition_e(const orc_params* p, const float* w, int n, const int32_t* j, const int32_t* e,
                             int N, double* logdet_out, double* quad_out);

/* Delta nu of one proposal from state z (j[0..N)), with either a Cholesky of both
 * states (mode 0) or eqs. (11)-(18) applied to Sigma^-1(z) built by successive births
 * (mode 1). kind: 0 birth of jp, 1 death of slot k, 2 update slot k -> jp. */
int orc_delta_nu(const orc_params* p, const float* w, int n, const int32_t* j, int N,
                 int kind, int k, int jp, int mode, double* dnu_out);
/* The same with PE components e[0..N) (NULL: all 0) and the component ep of the new PE. */
int orc_delta_nu_e(const orc_params* p, const float* w, int n, const int32_t* j, const int32_t* e, int N,
                   int kind, int k, int jp, int ep, int mode, double* dnu_out);

/* LucyDDM (Sec. 2.3): Lucy's iterative deconvolution of one waveform w[0..n) by the SER
 * sampled at the waveform's sample times, then the solution space and initial state.
 *  - q_out [n + L_V - 1] (may be NULL): q^(n_iter)(tau) for tau = -L_V+1 .. n-1;
 *  - z_out [z_cap]: grid indices tau R of the taus with q > thresh (at most z_cap; *n_z gets
 *    the number found, which may exceed z_cap);
 *  - *T_lo, *T_hi: the solution space [t_min - 4 ns, t_max + 4 ns] on the PE grid (T_hi
 *    exclusive), the whole window [0, n R) when no tau passes;
 *  - *t0_out: t_origin + t_min (NaN when none passes).
 * Returns L_V, or a negative error. */
int orc_lucyddm(const orc_params* p, const float* w, int n, double t_origin, int n_iter, double thresh,
                double* q_out, int32_t* z_out, int z_cap, int32_t* n_z, int32_t* T_lo, int32_t* T_hi,
                double* t0_out);

/* Run the chains of a batch; n_threads <= 0 uses one thread. trace: [n_waveforms*n_steps]
 * or NULL. Returns 0 or a negative error. */
int orc_run_batch(const orc_params* p, const orc_batch* b, int mode, int n_threads,
                  orc_summary* out, orc_trace* trace);

/* Run one chain (waveform 0 of b) and export its final state: PE list (n_cap entries) and
 * their components (n_cap entries, may be NULL), N, k0, Sigma^-1 (n*n, incremental mode
 * only), y (n), log|Sigma|. */
int orc_run_chain_state(const orc_params* p, const orc_batch* b, int mode,
                        orc_summary* out, orc_trace* trace, int32_t* list_out, int32_t* N_out,
                        int32_t* k0_out, double* sinv_out, double* y_out, double* logdet_out,
                        int32_t* e_out);

#ifdef __cplusplus
}
#endif
#endif

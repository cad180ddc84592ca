/*
 * fsmp_oracle.c -- plain FP64 CPU oracle of the FSMP chain (arXiv 2403.03156).
 *
 * TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs load this file's library. It shares no code with the CUDA path.
 *
 * The oracle follows the paper's steps in the paper's order and notation, with no
 * blocking, fusion or reordering:
 *   - tables: the SER of Sec. 3 and phi on the PE time grid;
 *   - definition mode: log p(w|z) from Sigma(z), U(z) of Eq. (mgauss) and a textbook
 *     Cholesky factorisation; Delta nu = log p(w|z') - log p(w|z), Eq. (delta-nu);
 *   - incremental mode: Sigma^-1 kept as a full n x n matrix, Delta nu by Eqs. (11),
 *     (DeltaU), (12), (16), (17), (18) literally (c = Sigma^-1 a, B = (Lambda^-1 + a^T c)^-1,
 *     Upsilon = c^T y + Lambda^-1 lambda), and the accept update Sigma^-1 -= c B c^T;
 *   - the chain: Gibbs step with MH on t0 (Sec. 2.4), then one RJMCMC jump chosen with
 *     probabilities J, J, 1-2J (birth / death / update, Sec. 2.4) and accepted with
 *     Eqs. (birth), (death), (update) and the posterior ratio above Eq. (delta-nu).
 *
 * Readings where the paper is silent (each one is restated at its use below):
 *   R1 PE times and t0 live on a grid of step g = grid_ns; the window's sample s sits at
 *      grid index s*R (R = dt_sample/g). A PE at grid index j contributes V[s*R - j].
 *   R2 The t0 prior is uniform on [t0_lo, t0_hi] (Eq. (t0prior)); a proposal outside is
 *      rejected. t0 and the PE times are shifted by rint(z * 1ns / g) grid steps,
 *      z ~ N(0,1) by Box-Muller, which keeps both proposals symmetric.
 *   R3 On the grid the Poisson prior of a multiset with multiplicities m_j is
 *      prod_j (lambda0 phi_j g)^m_j / m_j! (times constants), and h_j = phi_j g / Phi_T with
 *      Phi_T = sum_{j in T} phi_j g. Hence the birth log-ratio
 *      Delta nu + log lambda0 + log Phi_T - log(N+1), the death log-ratio its inverse, and
 *      the update log-ratio Delta nu + log phi(t+ - t0) - log phi(t- - t0).
 *   R4 From N = 0 only a birth is proposed and its ratio carries an extra J; a death from
 *      N = 1 carries 1/J (Sec. 2.4).
 *   R5 A birth at N = n_cap, an update leaving T, or a t0 move that puts a PE where
 *      phi = 0 is rejected. An update by zero grid steps is an accepted no-op.
 *   R6 Accept iff log u < log alpha (strict), u = ((x >> 11) + 0.5) 2^-53 from Philox4x64-10
 *      keyed by (seed, waveform index), counter (step, block, 0, 0); the 8 uniforms of a step
 *      are used as: u0,u1 t0 shift; u2 t0 accept; u3 jump type; u4 PE choice; u5,u6 update
 *      shift; u7 jump accept.
 *   R7 List discipline: birth appends at slot N, death moves slot N-1 into slot k, update
 *      overwrites slot k; the PE removed or moved is slot floor(u4 * N).
 *   R8 Charge summary: E[Q | z, w] = N mu_q + sigma_q^2 u^T Sigma^-1 y with u = sum_k a_k,
 *      the Gaussian posterior mean of the marginalised charges of Eq. (mgauss).
 *   R9 MCP model (n_mix > 1): a PE is (t_k, e_k). U and Sigma carry mu_{e_k} and
 *      sigma_{e_k}^2 per PE, Lambda = diag(-sigma_{e-}^2, sigma_{e+}^2) and
 *      lambda = (-mu_{e-}, mu_{e+}) (Appendix A.2). e+ ~ G (Sec. 2.4) is drawn for every
 *      birth and update from a ninth uniform u8 (Philox counter (step, 2, 0, 0), first
 *      output): the smallest e with G(0) + ... + G(e) > u8. The acceptances are Eq. (mcp)
 *      with the prior of Eq. (mcp-pzmu); an update with zero time shift and e+ = e- is the
 *      accepted no-op of R5, with e+ != e- it is a move. The charge summary of R8 becomes
 *      sum_k (mu_{e_k} + sigma_{e_k}^2 a_k^T Sigma^-1 y).
 *   R10 LucyDDM (Sec. 2.3) runs on the sample grid with the kernel v(m) = V(m dt) / S,
 *      m = 0 .. L_V-1, S = sum_m V(m dt) (the peak-normalised SER at the sample times, scaled
 *      to unit sum), on the data d(t) = max(w(t), 0) / S -- Lucy's method needs non-negative
 *      data, and the scaling makes q-hat a charge in units of the SER's. q-hat^0 is uniform
 *      with the sum of d; a ratio d / w^r with w^r = 0 is taken as 0. The printed index
 *      bounds of the w^r sum are garbled; w^r is the convolution sum over
 *      tau = t - L_V + 1 .. t. Each tau with q-hat > thresh gives one initial PE at grid index
 *      tau R; t0 starts at the first of them. A chain started from a given z (orc_batch.z_init)
 *      gives its PEs the mixture's most probable component.
 */
#include "fsmp_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI 6.283185307179586
#define ORC_LOG_2PI 1.8378770664093453
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_NOMEM (-2)

/* ------------------------------------------------------------------------------------
 * Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplications with a Weyl key schedule.
 * ---------------------------------------------------------------------------------- */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox_blocks(const uint64_t key[2], const uint64_t* ctrs, int n, uint64_t* out) {
  for (int i = 0; i < n; ++i) orc_philox4x64_10(ctrs + 4 * (size_t)i, key, out + 4 * (size_t)i);
}

static double orc_u01(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }

void orc_step_uniforms(uint64_t seed, uint64_t wf_index, uint64_t step, double u[8]) {
  uint64_t key[2] = {seed, wf_index};
  uint64_t c0[4] = {step, 0, 0, 0}, c1[4] = {step, 1, 0, 0};
  uint64_t o0[4], o1[4];
  orc_philox4x64_10(c0, key, o0);
  orc_philox4x64_10(c1, key, o1);
  for (int i = 0; i < 4; ++i) { u[i] = orc_u01(o0[i]); u[4 + i] = orc_u01(o1[i]); }
}

double orc_step_uniform_e(uint64_t seed, uint64_t wf_index, uint64_t step) {
  uint64_t key[2] = {seed, wf_index};
  uint64_t c2[4] = {step, 2, 0, 0};
  uint64_t o2[4];
  orc_philox4x64_10(c2, key, o2);
  return orc_u01(o2[0]);
}

/* ------------------------------------------------------------------------------------
 * SER and phi (Sec. 3).
 * ---------------------------------------------------------------------------------- */

/* The SER formula of Sec. 3: an ex-Gaussian shifted by 4 sigma,
 * (1/2tau) exp((sigma^2 - 2(t-4sigma)tau) / 2tau^2) (1 + Erf(-(sigma^2 - (t-4sigma)tau) / (sqrt2 sigma tau))).
 * 1 + Erf(-u) is evaluated as erfc(u) (the same function without the cancellation in the
 * left tail), and the product in log space so that exp() never overflows where erfc
 * vanishes. */
static double paper_ser(double t, double sigma, double tau) {
  double x = t - 4.0 * sigma;
  double expo = (sigma * sigma - 2.0 * x * tau) / (2.0 * tau * tau);
  double c = erfc((sigma * sigma - x * tau) / (sqrt(2.0) * sigma * tau));
  if (!(c > 0.0)) return 0.0;
  return exp(expo + log(c) - log(2.0 * tau));
}

/* The same ex-Gaussian density without the 4 sigma shift (phi of the configurations:
 * PE times are t0 plus an ex-Gaussian(sigma, tau) delay with Gaussian mean 0). */
static double exgauss_density(double x, double sigma, double tau) {
  double expo = (sigma * sigma - 2.0 * x * tau) / (2.0 * tau * tau);
  double c = erfc((sigma * sigma - x * tau) / (sqrt(2.0) * sigma * tau));
  if (!(c > 0.0)) return 0.0;
  return exp(expo + log(c) - log(2.0 * tau));
}

static int grid_ratio(const orc_params* p) {
  if (!(p->grid_ns > 0.0) || !(p->dt_sample_ns > 0.0)) return -1;
  double r = p->dt_sample_ns / p->grid_ns;
  long R = lround(r);
  if (R < 1 || R > 64 || fabs(r - (double)R) > 1e-9 * r) return -1;
  return (int)R;
}

/* Shape constants of the SER: the main pulse's grid peak and peak time, and for
 * ser_kind 1 the undershoot's own grid peak. The undershoot (reading for the "3%
 * undershoot" configuration) is a second, negative ex-Gaussian pulse of parameters
 * (ser_under_sigma, ser_under_tau), peak-normalised, scaled by ser_under_frac and started
 * at the main pulse's peak time. */
typedef struct { double main_peak, t_peak, under_peak; } ser_shape;

static double ser_scan_end(const orc_params* p) {
  double e = 8.0 * p->ser_sigma + 50.0 * p->ser_tau;
  if (p->ser_kind == 1) e += 8.0 * p->ser_under_sigma + 50.0 * p->ser_under_tau + e;
  return e;
}

static void ser_shape_init(const orc_params* p, ser_shape* sh) {
  double g = p->grid_ns;
  int m_end = (int)ceil(ser_scan_end(p) / g) + 1;
  sh->main_peak = 0.0; sh->t_peak = 0.0; sh->under_peak = 1.0;
  for (int m = 0; m < m_end; ++m) {
    double v = paper_ser(m * g, p->ser_sigma, p->ser_tau);
    if (v > sh->main_peak) { sh->main_peak = v; sh->t_peak = m * g; }
  }
  if (p->ser_kind == 1) {
    sh->under_peak = 0.0;
    for (int m = 0; m < m_end; ++m) {
      double v = paper_ser(m * g, p->ser_under_sigma, p->ser_under_tau);
      if (v > sh->under_peak) sh->under_peak = v;
    }
  }
}

static double ser_eval(const orc_params* p, const ser_shape* sh, double t) {
  double v = paper_ser(t, p->ser_sigma, p->ser_tau);
  if (p->ser_kind == 1) {
    double tu = t - sh->t_peak;
    double vu = tu >= 0.0 ? paper_ser(tu, p->ser_under_sigma, p->ser_under_tau) : 0.0;
    v = v / sh->main_peak - p->ser_under_frac * vu / sh->under_peak;
  }
  return v;
}

double orc_ser_raw(const orc_params* p, double t_ns) {
  ser_shape sh;
  ser_shape_init(p, &sh);
  return ser_eval(p, &sh, t_ns);
}

double orc_phi(const orc_params* p, double t) {
  if (fabs(t) > p->phi_support_ns) return 0.0;
  if (p->phi_kind == 0) return exgauss_density(t, p->phi_p1, p->phi_p2);
  /* LS two-exponential profile of Sec. 3 */
  if (t < 0.0) return 0.0;
  double t1 = p->phi_p1, t2 = p->phi_p2;
  return (t1 + t2) / (t2 * t2) * (1.0 - exp(-t / t1)) * exp(-t / t2);
}

int orc_ser_table(const orc_params* p, double* out, int max_len, double* peak_out) {
  int R = grid_ratio(p);
  if (R < 0 || !(p->ser_sigma > 0) || !(p->ser_tau > 0) || !(p->ser_eps > 0)) return ORC_ERR_INVALID;
  double g = p->grid_ns;
  ser_shape sh;
  ser_shape_init(p, &sh);
  int m_end = (int)ceil(ser_scan_end(p) / g) + 1;
  double peak = 0.0;
  for (int m = 0; m < m_end; ++m) {
    double v = ser_eval(p, &sh, m * g);
    if (v > peak) peak = v;
  }
  if (!(peak > 0.0)) return ORC_ERR_INVALID;
  int m_last = 0;
  for (int m = 0; m < m_end; ++m)
    if (fabs(ser_eval(p, &sh, m * g)) / peak >= p->ser_eps) m_last = m;
  int Lt = ((m_last + 1 + R - 1) / R) * R; /* whole samples: L_V = Lt / R */
  if (out) {
    if (Lt > max_len) return ORC_ERR_INVALID;
    for (int m = 0; m < Lt; ++m) out[m] = ser_eval(p, &sh, m * g) / peak;
  }
  if (peak_out) *peak_out = peak;
  return Lt;
}

/* ------------------------------------------------------------------------------------
 * Dense linear algebra (textbook, unblocked).
 * ---------------------------------------------------------------------------------- */

/* Cholesky-Banachiewicz: A (n x n, row-major, symmetric positive definite) -> lower L in
 * place. Returns 0, or -1 if a pivot is not positive. */
static int cholesky(double* A, int n) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return -1;
        A[i * n + i] = sqrt(s);
      } else {
        A[i * n + j] = s / A[j * n + j];
      }
    }
  }
  return 0;
}

/* Solve L x = b (forward) and L^T x = b (backward) for lower-triangular L. */
static void forward_sub(const double* L, int n, const double* b, double* x) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
    x[i] = s / L[i * n + i];
  }
}
static void backward_sub(const double* L, int n, const double* b, double* x) {
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/* ------------------------------------------------------------------------------------
 * The model: single-PE vectors a_j and the Gaussian marginal of Eq. (mgauss).
 * ---------------------------------------------------------------------------------- */
typedef struct {
  const orc_params* p;
  int R, Lt;
  double g;
  const double* V; /* peak-normalised SER table, Lt entries */
} model;

/* Charge model of a PE of component e (reading R9): N(mix_mu[e], mix_sigma[e]^2) of
 * Eq. (mcp-multi-norm), or the dynode N(mu_q, sigma_q^2) when n_mix = 0. */
static void charge_comp(const orc_params* p, int e, double* mu, double* s2) {
  if (p->n_mix > 0) {
    *mu = p->mix_mu[e];
    *s2 = p->mix_sigma[e] * p->mix_sigma[e];
  } else {
    *mu = p->mu_q;
    *s2 = p->sigma_q * p->sigma_q;
  }
}

/* e+ ~ G (Sec. 2.4): the smallest e whose cumulative probability exceeds u, else (rounding)
 * the last component with G > 0. 0 for the dynode model. */
static int draw_comp(const orc_params* p, double u) {
  if (p->n_mix <= 1) return 0;
  double cum = 0.0;
  int last = 0;
  for (int e = 0; e < p->n_mix; ++e) {
    if (p->mix_G[e] > 0.0) last = e;
    cum += p->mix_G[e];
    if (cum > u) return e;
  }
  return last;
}

/* a[w] = V(w*dt - t_j) on the grid (reading R1): V[w*R - j] inside the table, else 0. */
/* Samples of the window [0, n) in the support of a PE at grid index j (w R - j in [0, Lt)). */
static int support_count(const model* M, int n, int j) {
  int c = 0;
  for (int w = 0; w < n; ++w) {
    const int m = w * M->R - j;
    c += (m >= 0 && m < M->Lt);
  }
  return c;
}

/* Whether PEs at grid indices i and j share a sample of the window. */
static int supports_overlap(const model* M, int n, int i, int j) {
  for (int w = 0; w < n; ++w) {
    const int mi = w * M->R - i, mj = w * M->R - j;
    if (mi >= 0 && mi < M->Lt && mj >= 0 && mj < M->Lt) return 1;
  }
  return 0;
}

static void pe_vector(const model* M, int n, int j, double* a) {
  for (int w = 0; w < n; ++w) {
    int m = w * M->R - j;
    a[w] = (m >= 0 && m < M->Lt) ? M->V[m] : 0.0;
  }
}

/* log p(w|z) = -n/2 log 2pi - 1/2 log|Sigma| - 1/2 (w-U)^T Sigma^-1 (w-U), with
 * U_w = sum_k mu_{e_k} V(t_w - t_k) and Sigma = sum_k sigma_{e_k}^2 a_k a_k^T + sigma_eps^2 I
 * (Appendix A.1; per-PE components of Appendix A.2, e == NULL: all 0). Optionally returns
 * Sigma^-1 (w - U) in sinv_y. Returns NaN if Sigma is not positive definite. */
static double logp_def(const model* M, const float* wv, int n, const int32_t* j, const int32_t* e, int N,
                       double* logdet_out, double* quad_out, double* sinv_y) {
  const orc_params* p = M->p;
  double* S = (double*)calloc((size_t)n * n, sizeof(double));
  double* U = (double*)calloc((size_t)n, sizeof(double));
  double* a = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* x = (double*)malloc(sizeof(double) * n);
  double out = NAN;
  if (!S || !U || !a || !r || !x) goto done;
  for (int k = 0; k < N; ++k) {
    double mu, s2;
    charge_comp(p, e ? e[k] : 0, &mu, &s2);
    pe_vector(M, n, j[k], a);
    for (int w = 0; w < n; ++w) {
      U[w] += mu * a[w];
      for (int v = 0; v < n; ++v) S[w * n + v] += s2 * a[w] * a[v];
    }
  }
  for (int w = 0; w < n; ++w) S[w * n + w] += p->sigma_noise * p->sigma_noise;
  if (cholesky(S, n) != 0) goto done;
  double logdet = 0.0;
  for (int w = 0; w < n; ++w) logdet += 2.0 * log(S[w * n + w]);
  for (int w = 0; w < n; ++w) r[w] = (double)wv[w] - U[w];
  forward_sub(S, n, r, x);
  double quad = 0.0;
  for (int w = 0; w < n; ++w) quad += x[w] * x[w];
  if (sinv_y) backward_sub(S, n, x, sinv_y);
  if (logdet_out) *logdet_out = logdet;
  if (quad_out) *quad_out = quad;
  out = -0.5 * n * ORC_LOG_2PI - 0.5 * logdet - 0.5 * quad;
done:
  free(S); free(U); free(a); free(r); free(x);
  return out;
}

/* ------------------------------------------------------------------------------------
 * Incremental state: Sigma^-1 (full n x n), y = w - U(z), log|Sigma| (Appendix A.1).
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int n;
  double* Sinv;
  double* y;
  double logdet;
  /* scratch for one proposal */
  double *am, *ap, *cm, *cp;
  double B[2][2];
  double lam[2];
  double Linv[2];
} inc_state;

static int inc_init(inc_state* st, const orc_params* p, const float* wv, int n) {
  st->n = n;
  st->Sinv = (double*)calloc((size_t)n * n, sizeof(double));
  st->y = (double*)malloc(sizeof(double) * n);
  st->am = (double*)malloc(sizeof(double) * n);
  st->ap = (double*)malloc(sizeof(double) * n);
  st->cm = (double*)malloc(sizeof(double) * n);
  st->cp = (double*)malloc(sizeof(double) * n);
  if (!st->Sinv || !st->y || !st->am || !st->ap || !st->cm || !st->cp) return ORC_ERR_NOMEM;
  double s2 = p->sigma_noise * p->sigma_noise;
  for (int w = 0; w < n; ++w) {
    st->Sinv[w * n + w] = 1.0 / s2;
    st->y[w] = (double)wv[w];
  }
  st->logdet = n * log(s2);
  return 0;
}

static void inc_free(inc_state* st) {
  free(st->Sinv); free(st->y); free(st->am); free(st->ap); free(st->cm); free(st->cp);
}

/* Delta nu of the jump with single-PE vectors a_- = am, a_+ = ap (either may be all zero,
 * Eq. (11)): c = Sigma^-1 a, B = (Lambda^-1 + a^T c)^-1, Upsilon = c^T y + Lambda^-1 lambda,
 * Delta nu = 1/2 (Upsilon^T B Upsilon - lambda^T Lambda^-1 lambda + log|B Lambda^-1|)
 * (Eqs. (12), (16)-(18)), Lambda = diag(-sigma_{e-}^2, sigma_{e+}^2), lambda =
 * (-mu_{e-}, mu_{e+})^T (Eq. (DeltaU); Appendix A.2 for the components em, ep; the dynode
 * model has sigma_q, mu_q for both). Returns 0, or -1 if |B Lambda^-1| is not positive. */
static int inc_delta_nu(inc_state* st, const orc_params* p, int em, int ep, double* dnu) {
  int n = st->n;
  /* c = Sigma^-1 a; terms with a[v] == 0 contribute nothing and are skipped */
  for (int x = 0; x < n; ++x) { st->cm[x] = 0.0; st->cp[x] = 0.0; }
  for (int v = 0; v < n; ++v) {
    if (st->am[v] != 0.0)
      for (int x = 0; x < n; ++x) st->cm[x] += st->Sinv[x * n + v] * st->am[v];
    if (st->ap[v] != 0.0)
      for (int x = 0; x < n; ++x) st->cp[x] += st->Sinv[x * n + v] * st->ap[v];
  }
  double mu_m, s2_m, mu_p, s2_p;
  charge_comp(p, em, &mu_m, &s2_m);
  charge_comp(p, ep, &mu_p, &s2_p);
  st->Linv[0] = -1.0 / s2_m; /* Lambda^-1 (diagonal) */
  st->Linv[1] = 1.0 / s2_p;
  const double* Linv = st->Linv;
  st->lam[0] = -mu_m;
  st->lam[1] = mu_p;
  /* a^T c = a^T Sigma^-1 a is symmetric because Sigma^-1 is: its off-diagonal is computed
   * once (a_-^T c_+) and used for both entries, so B below is exactly symmetric. */
  double atc[2][2] = {{0, 0}, {0, 0}};
  double cty[2] = {0, 0};
  for (int x = 0; x < n; ++x) {
    atc[0][0] += st->am[x] * st->cm[x];
    atc[0][1] += st->am[x] * st->cp[x];
    atc[1][1] += st->ap[x] * st->cp[x];
    cty[0] += st->cm[x] * st->y[x];
    cty[1] += st->cp[x] * st->y[x];
  }
  atc[1][0] = atc[0][1];
  double P00 = Linv[0] + atc[0][0], P01 = atc[0][1], P10 = atc[1][0], P11 = Linv[1] + atc[1][1];
  double detP = P00 * P11 - P01 * P10;
  st->B[0][0] = P11 / detP;
  st->B[0][1] = -P01 / detP;
  st->B[1][0] = -P10 / detP;
  st->B[1][1] = P00 / detP;
  double Ups[2] = {cty[0] + Linv[0] * st->lam[0], cty[1] + Linv[1] * st->lam[1]};
  double UBU = Ups[0] * (st->B[0][0] * Ups[0] + st->B[0][1] * Ups[1]) +
               Ups[1] * (st->B[1][0] * Ups[0] + st->B[1][1] * Ups[1]);
  double lLl = st->lam[0] * Linv[0] * st->lam[0] + st->lam[1] * Linv[1] * st->lam[1];
  double detB = st->B[0][0] * st->B[1][1] - st->B[0][1] * st->B[1][0];
  double detBL = detB * Linv[0] * Linv[1];
  if (!(detBL > 0.0) || !isfinite(detBL)) return -1;
  *dnu = 0.5 * (UBU - lLl + log(detBL));
  return 0;
}

/* Accept: Sigma'^-1 = Sigma^-1 - c B c^T (Eq. (12)), y' = y - a lambda (Eq. (DeltaU)),
 * log|Sigma'| = log|Sigma| + Delta T with Delta T = -log|B Lambda^-1| (Eq. (17)).
 * Sigma'^-1 is symmetric: each entry (x, v), v <= x, is computed once and mirrored. Without
 * this, rounding leaves an antisymmetric part that the recursion amplifies geometrically
 * over repeated update jumps. */
static void inc_accept(inc_state* st, const orc_params* p) {
  int n = st->n;
  for (int x = 0; x < n; ++x) {
    double b0 = st->B[0][0] * st->cm[x] + st->B[0][1] * st->cp[x];
    double b1 = st->B[1][0] * st->cm[x] + st->B[1][1] * st->cp[x];
    for (int v = 0; v <= x; ++v) {
      double e = st->Sinv[x * n + v] - (b0 * st->cm[v] + b1 * st->cp[v]);
      st->Sinv[x * n + v] = e;
      st->Sinv[v * n + x] = e;
    }
  }
  for (int x = 0; x < n; ++x) st->y[x] -= st->am[x] * st->lam[0] + st->ap[x] * st->lam[1];
  (void)p;
  double detB = st->B[0][0] * st->B[1][1] - st->B[0][1] * st->B[1][0];
  double detBL = detB * st->Linv[0] * st->Linv[1];
  st->logdet += -log(detBL);
}

/* ------------------------------------------------------------------------------------
 * One chain.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  const orc_params* p;
  const model* M;
  const float* w;
  int n;
  double lambda0, t_origin;
  int T_lo, T_hi, k0_lo, k0_hi, k0_init;
  uint64_t seed, wf_index;
  int n_steps, burn_in, mode;
  const uint8_t* forced;
  double* occ;
  int occ_width;
  double* occ_e;
  const int32_t* z_init; /* initial PE grid indices (NULL: empty) */
  int n_init;
} chain_in;

typedef struct {
  int d_min, d_max;
  double* phi;    /* phi((d) g), d in [d_min, d_max] */
  double* logphi;
  double* Phi_T;  /* Phi_T(k0) for k0 in [k0_lo, k0_hi], NaN until first use */
} chain_tabs;

static double tab_phi(const chain_tabs* t, int d) {
  if (d < t->d_min || d > t->d_max) return 0.0;
  return t->phi[d - t->d_min];
}
static double tab_logphi(const chain_tabs* t, int d) {
  if (d < t->d_min || d > t->d_max) return -INFINITY;
  return t->logphi[d - t->d_min];
}

/* Phi_T(t0) = sum over grid points j in T of phi(j g - t0) g (the normaliser of h, Sec. 2.4). */
static double tab_Phi_T(const chain_in* c, chain_tabs* t, int k0) {
  double* slot = &t->Phi_T[k0 - c->k0_lo];
  if (isnan(*slot)) {
    double s = 0.0;
    for (int j = c->T_lo; j < c->T_hi; ++j) s += tab_phi(t, j - k0) * c->M->g;
    *slot = s;
  }
  return *slot;
}

/* log G(e) of the MCP model (reading R9); 0 for the dynode model. */
static double log_G(const orc_params* p, int e) { return p->n_mix > 1 ? log(p->mix_G[e]) : 0.0; }

static int run_chain(const chain_in* c, orc_summary* out, orc_trace* trace, int32_t* list_out,
                     int32_t* N_out, int32_t* k0_out, double* sinv_out, double* y_out,
                     double* logdet_out, int32_t* e_out) {
  const orc_params* p = c->p;
  const model* M = c->M;
  const int n = c->n;
  const double g = M->g;
  const double inv_g = 1.0 / g;
  int rc = 0;
  memset(out, 0, sizeof(*out));

  chain_tabs tb;
  tb.d_min = c->T_lo - c->k0_hi;
  tb.d_max = c->T_hi - 1 - c->k0_lo;
  int nd = tb.d_max - tb.d_min + 1;
  tb.phi = (double*)malloc(sizeof(double) * (nd > 0 ? nd : 1));
  tb.logphi = (double*)malloc(sizeof(double) * (nd > 0 ? nd : 1));
  tb.Phi_T = (double*)malloc(sizeof(double) * (c->k0_hi - c->k0_lo + 1));
  int32_t* list = (int32_t*)calloc((size_t)p->n_cap + 1, sizeof(int32_t));
  int32_t* list_e = (int32_t*)calloc((size_t)p->n_cap + 1, sizeof(int32_t)); /* components */
  int32_t* zprop_e = (int32_t*)calloc((size_t)p->n_cap + 1, sizeof(int32_t));
  double* av = (double*)malloc(sizeof(double) * n);
  double* uvec = (double*)malloc(sizeof(double) * n);
  double* svec = (double*)malloc(sizeof(double) * n);
  int32_t* zprop = (int32_t*)malloc(sizeof(int32_t) * (p->n_cap + 1));
  inc_state st;
  memset(&st, 0, sizeof(st));
  if (!tb.phi || !tb.logphi || !tb.Phi_T || !list || !list_e || !zprop_e || !av || !uvec || !svec || !zprop) {
    rc = ORC_ERR_NOMEM;
    goto done;
  }
  for (int d = tb.d_min; d <= tb.d_max; ++d) {
    double ph = orc_phi(p, d * g);
    tb.phi[d - tb.d_min] = ph;
    tb.logphi[d - tb.d_min] = ph > 0.0 ? log(ph) : -INFINITY;
  }
  for (int k = 0; k <= c->k0_hi - c->k0_lo; ++k) tb.Phi_T[k] = NAN;

  if (c->mode == ORC_MODE_INCREMENTAL && !p->prior_only) {
    if (inc_init(&st, p, c->w, n) != 0) { rc = ORC_ERR_NOMEM; goto done; }
  }
  int N = 0;
  int k0 = c->k0_init;
  /* initial state: empty z, or the given one (the LucyDDM state of Sec. 2.3, reading R10):
   * at most n_cap PEs, each of the mixture's most probable component; Sigma^-1 built from the
   * empty state by successive births (Eq. (12) with a_- = 0) */
  if (c->z_init) {
    int e0 = 0;
    for (int e = 1; e < p->n_mix; ++e)
      if (p->mix_G[e] > p->mix_G[e0]) e0 = e;
    N = c->n_init;
    if (N > p->n_cap) { N = p->n_cap; out->status |= ORC_ST_CAPACITY; }
    for (int k = 0; k < N; ++k) { list[k] = c->z_init[k]; list_e[k] = e0; }
    if (c->mode == ORC_MODE_INCREMENTAL && !p->prior_only)
      for (int k = 0; k < N; ++k) {
        double d;
        for (int x = 0; x < n; ++x) st.am[x] = 0.0;
        pe_vector(M, n, list[k], st.ap);
        if (inc_delta_nu(&st, p, e0, e0, &d) != 0) { rc = ORC_ERR_INVALID; goto done; }
        inc_accept(&st, p);
      }
  }
  double logp_cur = 0.0;
  if (c->mode == ORC_MODE_DEFINITION && !p->prior_only)
    logp_cur = logp_def(M, c->w, n, list, list_e, N, NULL, NULL, NULL);

  double sN = 0, sN2 = 0, st0 = 0, st02 = 0, sQ = 0, sQ2 = 0, sWt = 0, sWt2 = 0, sWe = 0, sWe2 = 0;
  double* hist = (double*)calloc((size_t)p->n_cap + 1, sizeof(double));
  double* wbuf = (double*)malloc(sizeof(double) * ((size_t)p->n_cap + 1));
  double* wbuf_e = (double*)malloc(sizeof(double) * ((size_t)p->n_cap + 1));
  int q_valid = 0;
  double q_cur = 0.0;
  const double logJ = log(p->jump_J);

  for (int step = 0; step < c->n_steps; ++step) {
    double u[8];
    orc_step_uniforms(c->seed, c->wf_index, (uint64_t)step, u);
    orc_trace tr;
    tr.la0 = NAN; tr.lu0 = NAN; tr.la = NAN; tr.lu = NAN; tr.dnu = NAN;
    tr.flags = 0;
    uint8_t forced = c->forced ? c->forced[step] : 0;
    /* component of a born or updated PE, e+ ~ G (reading R9) */
    const int ep = p->n_mix > 1 ? draw_comp(p, orc_step_uniform_e(c->seed, c->wf_index, (uint64_t)step)) : 0;

    /* ---- Gibbs part 1: MH on t0 given z (Sec. 2.4, reading R2) ---- */
    if (p->sample_t0) {
      tr.flags |= ORC_F_T0_PROPOSED;
      out->prop_t0++;
      double z1 = sqrt(-2.0 * log(u[0])) * cos(ORC_TWO_PI * u[1]);
      long D = (long)rint(z1 * inv_g);
      long k0p = k0 + D;
      double la0;
      if (D == 0) {
        la0 = 0.0;
      } else if (k0p < c->k0_lo || k0p > c->k0_hi) {
        la0 = -INFINITY; /* outside the uniform prior of Eq. (t0prior) */
      } else {
        /* log p(t0'|z) - log p(t0|z) = sum_k [log phi(t_k - t0') - log phi(t_k - t0)] */
        la0 = 0.0;
        for (int k = 0; k < N; ++k) {
          double lnew = tab_logphi(&tb, list[k] - (int)k0p);
          if (lnew == -INFINITY) { la0 = -INFINITY; break; }
          la0 += lnew - tab_logphi(&tb, list[k] - k0);
        }
      }
      double lu0 = log(u[2]);
      int acc0 = lu0 < la0;
      if (c->forced) {
        int f = forced & 1;
        if (f != acc0) { tr.flags |= ORC_F_T0_DISAGREE; out->status |= ORC_ST_DISAGREE; }
        acc0 = f;
      }
      if (acc0) {
        tr.flags |= ORC_F_T0_ACCEPTED;
        out->acc_t0++;
        k0 = (int)k0p;
      }
      tr.la0 = la0; tr.lu0 = lu0;
    }

    /* ---- Gibbs part 2: one RJMCMC jump on z (Sec. 2.4) ---- */
    int jump;
    if (N == 0) jump = ORC_JUMP_BIRTH;
    else if (u[3] < p->jump_J) jump = ORC_JUMP_BIRTH;
    else if (u[3] < 2.0 * p->jump_J) jump = ORC_JUMP_DEATH;
    else jump = ORC_JUMP_UPDATE;
    out->prop[jump]++;

    double la = -INFINITY, dnu = NAN;
    int noop = 0, k = -1, jp = -1, valid = 0;
    int Nprop = N;
    if (jump == ORC_JUMP_BIRTH) {
      double Phi = tab_Phi_T(c, &tb, k0);
      if (N >= p->n_cap) {
        out->status |= ORC_ST_CAPACITY; /* reading R5 */
      } else if (Phi > 0.0) {
        /* t_+ ~ h(t) = phi(t - t0) / Phi_T: the first grid point whose cumulative mass
         * exceeds u4 Phi_T */
        double target = u[4] * Phi, cum = 0.0;
        int jlast = -1;
        for (int j = c->T_lo; j < c->T_hi; ++j) {
          double ph = tab_phi(&tb, j - k0);
          if (ph > 0.0) jlast = j;
          cum += ph * g;
          if (cum > target) { jp = j; break; }
        }
        if (jp < 0) jp = jlast;
        memcpy(zprop, list, sizeof(int32_t) * N);
        memcpy(zprop_e, list_e, sizeof(int32_t) * N);
        zprop[N] = jp;
        zprop_e[N] = ep;
        Nprop = N + 1;
        valid = 1;
      }
    } else {
      k = (int)floor(u[4] * N);
      if (k >= N) k = N - 1;
      if (jump == ORC_JUMP_DEATH) {
        memcpy(zprop, list, sizeof(int32_t) * N);
        memcpy(zprop_e, list_e, sizeof(int32_t) * N);
        zprop[k] = list[N - 1];
        zprop_e[k] = list_e[N - 1];
        Nprop = N - 1;
        valid = 1;
      } else {
        double z2 = sqrt(-2.0 * log(u[5])) * cos(ORC_TWO_PI * u[6]);
        long D = (long)rint(z2 * inv_g);
        jp = list[k] + (int)D;
        if (D == 0 && ep == list_e[k]) {
          noop = 1; /* readings R5, R9: an accepted no-op */
          la = 0.0;
        } else if (jp < c->T_lo || jp >= c->T_hi || tab_logphi(&tb, jp - k0) == -INFINITY) {
          la = -INFINITY;
        } else {
          memcpy(zprop, list, sizeof(int32_t) * N);
          memcpy(zprop_e, list_e, sizeof(int32_t) * N);
          zprop[k] = jp;
          zprop_e[k] = ep;
          Nprop = N;
          valid = 1;
        }
      }
    }

    /* the words the method moves to score this proposal (orc_summary.alg_words) */
    int np_w = 0, sp_len = 0, sm_len = 0;
    if (valid && jump != ORC_JUMP_DEATH) {
      sp_len = support_count(M, n, jp);
      for (int q = 0; q < N; ++q) np_w += supports_overlap(M, n, list[q], jp);
      out->alg_words += N + 2.0 * np_w + 2.0 * sp_len + (double)np_w * np_w + np_w;
    }
    if (valid && jump != ORC_JUMP_BIRTH) {
      sm_len = support_count(M, n, list[k]);
      out->alg_words += 2.0;
    }

    double logp_new = 0.0;
    if (valid) {
      int ok = 1;
      if (p->prior_only) {
        dnu = 0.0;
      } else if (c->mode == ORC_MODE_DEFINITION) {
        logp_new = logp_def(M, c->w, n, zprop, zprop_e, Nprop, NULL, NULL, NULL);
        dnu = logp_new - logp_cur; /* Eq. (delta-nu) */
        if (!isfinite(dnu)) { ok = 0; out->status |= ORC_ST_NONFINITE; }
      } else {
        if (jump == ORC_JUMP_BIRTH) { for (int w = 0; w < n; ++w) st.am[w] = 0.0; pe_vector(M, n, jp, st.ap); }
        else if (jump == ORC_JUMP_DEATH) { pe_vector(M, n, list[k], st.am); for (int w = 0; w < n; ++w) st.ap[w] = 0.0; }
        else { pe_vector(M, n, list[k], st.am); pe_vector(M, n, jp, st.ap); }
        /* components of a_- and a_+; the absent one of a birth or death does not enter */
        const int e_minus = jump == ORC_JUMP_BIRTH ? ep : list_e[k];
        const int e_plus = jump == ORC_JUMP_DEATH ? e_minus : ep;
        if (inc_delta_nu(&st, p, e_minus, e_plus, &dnu) != 0) { ok = 0; out->status |= ORC_ST_BADDET; }
        else if (!isfinite(dnu)) { ok = 0; out->status |= ORC_ST_NONFINITE; }
      }
      if (ok) {
        double Phi = tab_Phi_T(c, &tb, k0);
        /* Eq. (mcp): the prior of Eq. (mcp-pzmu) carries G(e) per PE and the proposal draws
         * e+ ~ G, so a birth gains G(e+) / G(e+), a death G(e-) / G(e-) and an update
         * G(e+) G(e-) / (G(e-) G(e+)); the terms are kept as the paper writes them */
        if (jump == ORC_JUMP_BIRTH)
          la = dnu + log(c->lambda0) + log(Phi) - log((double)(N + 1)) + (N == 0 ? logJ : 0.0) + log_G(p, ep) -
               log_G(p, ep);
        else if (jump == ORC_JUMP_DEATH)
          la = dnu - log(c->lambda0) - log(Phi) + log((double)N) - (N == 1 ? logJ : 0.0) - log_G(p, list_e[k]) +
               log_G(p, list_e[k]);
        else
          la = dnu + tab_logphi(&tb, jp - k0) - tab_logphi(&tb, list[k] - k0) + log_G(p, ep) - log_G(p, list_e[k]) +
               log_G(p, list_e[k]) - log_G(p, ep);
      } else {
        la = -INFINITY;
      }
    }
    double lu = log(u[7]);
    int acc = lu < la;
    if (c->forced) {
      int f = (forced >> 1) & 1;
      if (f != acc) { tr.flags |= ORC_F_DISAGREE; out->status |= ORC_ST_DISAGREE; }
      acc = f;
      if (acc && !valid && !noop) acc = 0; /* nothing to apply */
    }
    if (acc) {
      tr.flags |= ORC_F_ACCEPTED;
      if (noop) {
        tr.flags |= ORC_F_NOOP;
      } else {
        out->acc[jump]++;
        {
          const double Nout = N + (jump == ORC_JUMP_BIRTH ? 1 : (jump == ORC_JUMP_DEATH ? -1 : 0));
          out->alg_words += (double)N * np_w + Nout * (Nout + 1.0) + 2.0 * Nout;
          if (jump != ORC_JUMP_BIRTH) out->alg_words += 2.0 * sm_len + N;
          if (jump != ORC_JUMP_DEATH) out->alg_words += 2.0 * sp_len;
        }
        if (c->mode == ORC_MODE_INCREMENTAL && !p->prior_only) inc_accept(&st, p);
        if (c->mode == ORC_MODE_DEFINITION) logp_cur = logp_new;
        if (jump == ORC_JUMP_BIRTH) { list[N] = jp; list_e[N] = ep; N++; }
        else if (jump == ORC_JUMP_DEATH) { list[k] = list[N - 1]; list_e[k] = list_e[N - 1]; N--; }
        else { list[k] = jp; list_e[k] = ep; }
        q_valid = 0;
      }
    }
    tr.la = la; tr.lu = lu; tr.dnu = dnu;
    tr.N = N; tr.k0 = k0; tr.jump = jump;
    /* the Wasserstein scalars of the new state (convergence check of Sec. 3.2) */
    for (int kk = 0; kk < N; ++kk) { wbuf[kk] = list[kk] * g; wbuf_e[kk] = list_e[kk]; }
    tr.wt = orc_pe_wasserstein(wbuf, N);
    tr.we = orc_pe_wasserstein(wbuf_e, N);
    if (trace) trace[step] = tr;

    /* ---- summaries after burn-in (reading R8 for the charge) ---- */
    if (step >= c->burn_in) {
      if (!q_valid) {
        if (p->prior_only) {
          q_cur = 0.0;
          for (int kk = 0; kk < N; ++kk) {
            double mu, s2;
            charge_comp(p, list_e[kk], &mu, &s2);
            q_cur += mu;
          }
        } else {
          if (c->mode == ORC_MODE_INCREMENTAL) {
            for (int x = 0; x < n; ++x) {
              double s = 0.0;
              for (int v = 0; v < n; ++v) s += st.Sinv[x * n + v] * st.y[v];
              svec[x] = s;
            }
          } else {
            logp_def(M, c->w, n, list, list_e, N, NULL, NULL, svec);
          }
          /* sum_k (mu_{e_k} + sigma_{e_k}^2 a_k^T Sigma^-1 y) (readings R8, R9) */
          q_cur = 0.0;
          for (int kk = 0; kk < N; ++kk) {
            double mu, s2;
            charge_comp(p, list_e[kk], &mu, &s2);
            pe_vector(M, n, list[kk], av);
            double as = 0.0;
            for (int x = 0; x < n; ++x) as += av[x] * svec[x];
            q_cur += mu + s2 * as;
          }
        }
        q_valid = 1;
      }
      double t0ns = c->t_origin + k0 * g;
      sN += N; sN2 += (double)N * N;
      if (N >= 0 && N <= p->n_cap) hist[N] += 1.0;
      st0 += t0ns; st02 += t0ns * t0ns;
      sWt += tr.wt; sWt2 += tr.wt * tr.wt;
      sWe += tr.we; sWe2 += tr.we * tr.we;
      sQ += q_cur; sQ2 += q_cur * q_cur;
      if (c->occ)
        for (int kk = 0; kk < N; ++kk) {
          int col = list[kk] - c->T_lo;
          if (col >= 0 && col < c->occ_width) c->occ[col] += 1.0;
        }
      if (c->occ_e)
        for (int kk = 0; kk < N; ++kk) c->occ_e[list_e[kk]] += 1.0;
    }
  }

  {
    int ns = c->n_steps - c->burn_in;
    if (ns < 0) ns = 0;
    out->n_samples = ns;
    double inv = ns > 0 ? 1.0 / ns : NAN;
    out->mean_N = sN * inv; out->var_N = sN2 * inv - out->mean_N * out->mean_N;
    out->mean_t0 = st0 * inv; out->var_t0 = st02 * inv - out->mean_t0 * out->mean_t0;
    out->mean_Q = sQ * inv; out->var_Q = sQ2 * inv - out->mean_Q * out->mean_Q;
    out->mean_wt = sWt * inv; out->var_wt = sWt2 * inv - out->mean_wt * out->mean_wt;
    out->mean_we = sWe * inv; out->var_we = sWe2 * inv - out->mean_we * out->mean_we;
    out->N_final = N;
    out->k0_final = k0;
    out->lambda_hat = ns > 0 ? orc_lambda_mle(hist, p->n_cap, c->lambda0) : NAN;
    if (c->occ && ns > 0)
      for (int col = 0; col < c->occ_width; ++col) c->occ[col] *= inv;
    if (c->occ_e && ns > 0)
      for (int e = 0; e < (p->n_mix > 1 ? p->n_mix : 1); ++e) c->occ_e[e] *= inv;
    if (p->prior_only) {
      out->logL = NAN; out->logdet = NAN;
    } else if (c->mode == ORC_MODE_INCREMENTAL) {
      double quad = 0.0;
      for (int x = 0; x < n; ++x) {
        double s = 0.0;
        for (int v = 0; v < n; ++v) s += st.Sinv[x * n + v] * st.y[v];
        quad += st.y[x] * s;
      }
      out->logdet = st.logdet;
      out->logL = -0.5 * n * ORC_LOG_2PI - 0.5 * st.logdet - 0.5 * quad;
    } else {
      double ld = 0.0;
      out->logL = logp_def(M, c->w, n, list, list_e, N, &ld, NULL, NULL);
      out->logdet = ld;
    }
    if (list_out) memcpy(list_out, list, sizeof(int32_t) * N);
    if (e_out) memcpy(e_out, list_e, sizeof(int32_t) * N);
    if (N_out) *N_out = N;
    if (k0_out) *k0_out = k0;
    if (c->mode == ORC_MODE_INCREMENTAL && !p->prior_only) {
      if (sinv_out) memcpy(sinv_out, st.Sinv, sizeof(double) * n * n);
      if (y_out) memcpy(y_out, st.y, sizeof(double) * n);
      if (logdet_out) *logdet_out = st.logdet;
    }
    free(hist);
  }
  free(wbuf);
  free(wbuf_e);
done:
  free(tb.phi); free(tb.logphi); free(tb.Phi_T); free(list); free(list_e); free(zprop_e);
  free(av); free(uvec); free(svec); free(zprop);
  if (st.Sinv) inc_free(&st);
  return rc;
}

/* ------------------------------------------------------------------------------------
 * LucyDDM (Sec. 2.3, reading R10).
 * ---------------------------------------------------------------------------------- */
static int lucyddm(const model* M, const float* wv, int n, double t_origin, int n_iter, double thresh,
                   double* q_out, int32_t* z_out, int z_cap, int32_t* n_z, int32_t* T_lo, int32_t* T_hi,
                   double* t0_out) {
  const int LV = M->Lt / M->R, nq = n + LV - 1;
  double* v = (double*)malloc(sizeof(double) * LV);
  double* d = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * nq);
  double* wr = (double*)malloc(sizeof(double) * n);
  double* ratio = (double*)malloc(sizeof(double) * n);
  if (!v || !d || !q || !wr || !ratio) {
    free(v); free(d); free(q); free(wr); free(ratio);
    return ORC_ERR_NOMEM;
  }
  /* kernel: the SER at the sample times, scaled to unit sum */
  double S = 0.0;
  for (int m = 0; m < LV; ++m) S += M->V[m * M->R];
  for (int m = 0; m < LV; ++m) v[m] = M->V[m * M->R] / S;
  double dsum = 0.0;
  for (int t = 0; t < n; ++t) {
    d[t] = wv[t] > 0.0f ? (double)wv[t] / S : 0.0;
    dsum += d[t];
  }
  /* q[i] is q-hat(tau) at tau = i - (LV - 1); q-hat^0 uniform with the sum of d */
  for (int i = 0; i < nq; ++i) q[i] = dsum / nq;
  for (int r = 0; r < n_iter; ++r) {
    /* w^r(t) = sum_{tau = t - LV + 1}^{t} q-hat(tau) v(t - tau) */
    for (int t = 0; t < n; ++t) {
      double s = 0.0;
      for (int m = 0; m < LV; ++m) s += q[t - m + (LV - 1)] * v[m];
      wr[t] = s;
      ratio[t] = s > 0.0 ? d[t] / s : 0.0;
    }
    /* q-hat(tau) *= sum_{t = max(tau, 0)}^{min(n - 1, tau + LV - 1)} ratio(t) v(t - tau) */
    for (int i = 0; i < nq; ++i) {
      const int tau = i - (LV - 1);
      double s = 0.0;
      for (int m = 0; m < LV; ++m) {
        const int t = tau + m;
        if (t >= 0 && t < n) s += ratio[t] * v[m];
      }
      q[i] *= s;
    }
  }
  if (q_out) memcpy(q_out, q, sizeof(double) * nq);
  /* initial PEs, solution space and t0 (Sec. 2.3) */
  int cnt = 0, tmin = 0, tmax = 0;
  for (int i = 0; i < nq; ++i) {
    if (!(q[i] > thresh)) continue;
    const int tau = i - (LV - 1);
    if (cnt == 0) tmin = tau;
    tmax = tau;
    if (cnt < z_cap) z_out[cnt] = tau * M->R;
    ++cnt;
  }
  *n_z = cnt;
  if (cnt == 0) {
    *T_lo = 0;
    *T_hi = n * M->R;
    *t0_out = NAN;
  } else {
    const double dt = M->p->dt_sample_ns, g = M->g;
    *T_lo = (int32_t)floor((tmin * dt - 4.0) / g + 1e-9);
    *T_hi = (int32_t)ceil((tmax * dt + 4.0) / g - 1e-9) + 1;
    *t0_out = t_origin + tmin * dt;
  }
  free(v); free(d); free(q); free(wr); free(ratio);
  return LV;
}

/* ------------------------------------------------------------------------------------
 * Batch plumbing.
 * ---------------------------------------------------------------------------------- */
static int check_params(const orc_params* p) {
  if (grid_ratio(p) < 0) return ORC_ERR_INVALID;
  if (!(p->sigma_noise > 0) || !(p->sigma_q > 0) || !(p->jump_J > 0) || !(p->jump_J <= 0.5)) return ORC_ERR_INVALID;
  if (p->n_cap < 1 || !(p->phi_support_ns > 0)) return ORC_ERR_INVALID;
  if (!(p->t0_hi >= p->t0_lo)) return ORC_ERR_INVALID;
  if (p->n_mix < 0 || p->n_mix > ORC_MAX_MIX) return ORC_ERR_INVALID;
  if (p->n_mix > 0) {
    double sum = 0.0;
    for (int e = 0; e < p->n_mix; ++e) {
      if (!(p->mix_G[e] >= 0.0) || !(p->mix_sigma[e] > 0.0) || !isfinite(p->mix_mu[e])) return ORC_ERR_INVALID;
      sum += p->mix_G[e];
    }
    if (!(fabs(sum - 1.0) <= 1e-9)) return ORC_ERR_INVALID; /* G is a distribution (Appendix A.2) */
  }
  return 0;
}

/* Prior range of t0 on the grid (reading R2): ceil / floor with a 1e-9 grid-step slack
 * so that bounds that are exact multiples of g survive rounding of the division. */
static int make_chain_in(const orc_params* p, const model* M, const orc_batch* b, int i, int mode,
                         chain_in* c) {
  int32_t off0 = b->offsets[i], off1 = b->offsets[i + 1];
  c->p = p; c->M = M;
  c->w = b->samples + off0;
  c->n = off1 - off0;
  if (c->n < 1) return ORC_ERR_INVALID;
  c->lambda0 = b->lambda0[i];
  if (!(c->lambda0 > 0)) return ORC_ERR_INVALID;
  c->t_origin = b->t_origin_ns ? b->t_origin_ns[i] : 0.0;
  c->T_lo = b->T_lo ? b->T_lo[i] : 0;
  c->T_hi = b->T_hi ? b->T_hi[i] : c->n * M->R;
  if (c->T_hi <= c->T_lo) return ORC_ERR_INVALID;
  double g = M->g;
  c->k0_lo = (int)ceil((p->t0_lo - c->t_origin) / g - 1e-9);
  c->k0_hi = (int)floor((p->t0_hi - c->t_origin) / g + 1e-9);
  if (c->k0_hi < c->k0_lo) return ORC_ERR_INVALID;
  if (b->t0_init && !isnan(b->t0_init[i])) {
    double kk = rint((b->t0_init[i] - c->t_origin) / g);
    if (kk < c->k0_lo) kk = c->k0_lo;
    if (kk > c->k0_hi) kk = c->k0_hi;
    c->k0_init = (int)kk;
  } else {
    c->k0_init = c->k0_lo + (c->k0_hi - c->k0_lo) / 2;
  }
  c->seed = b->seed;
  c->wf_index = b->wf_ids ? b->wf_ids[i] : b->index_base + (uint64_t)i;
  c->n_steps = b->n_steps;
  c->burn_in = b->burn_in;
  c->mode = mode;
  c->forced = b->forced ? b->forced + (size_t)i * b->n_steps : NULL;
  c->occ = b->occ ? b->occ + (size_t)i * b->occ_width : NULL;
  c->occ_width = b->occ_width;
  c->occ_e = b->occ_e ? b->occ_e + (size_t)i * (p->n_mix > 1 ? p->n_mix : 1) : NULL;
  c->z_init = NULL;
  c->n_init = 0;
  if (b->z_init) {
    if (!b->n_init || b->n_init[i] < 0 || b->n_init[i] > b->z_stride) return ORC_ERR_INVALID;
    c->z_init = b->z_init + (size_t)i * b->z_stride;
    c->n_init = b->n_init[i];
  }
  return 0;
}

typedef struct {
  const orc_params* p;
  const model* M;
  const orc_batch* b;
  int mode, tid, nthreads;
  orc_summary* out;
  orc_trace* trace;
  int rc;
} worker_arg;

static void* worker(void* arg) {
  worker_arg* a = (worker_arg*)arg;
  a->rc = 0;
  for (int i = a->tid; i < a->b->n_waveforms; i += a->nthreads) {
    chain_in c;
    int rc = make_chain_in(a->p, a->M, a->b, i, a->mode, &c);
    if (rc == 0)
      rc = run_chain(&c, &a->out[i], a->trace ? a->trace + (size_t)i * a->b->n_steps : NULL,
                     NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    if (rc != 0) a->rc = rc;
  }
  return NULL;
}

static int build_model(const orc_params* p, model* M, double** Vbuf) {
  int rc = check_params(p);
  if (rc) return rc;
  int Lt = orc_ser_table(p, NULL, 0, NULL);
  if (Lt < 0) return Lt;
  *Vbuf = (double*)malloc(sizeof(double) * Lt);
  if (!*Vbuf) return ORC_ERR_NOMEM;
  orc_ser_table(p, *Vbuf, Lt, NULL);
  M->p = p; M->R = grid_ratio(p); M->Lt = Lt; M->g = p->grid_ns; M->V = *Vbuf;
  return 0;
}

/* l(lambda) = -lambda + log sum_N h[N] (lambda / lambda0)^N, the log of Eq. (reduce-mu0) up to
 * a constant, evaluated as a log-sum-exp over the N with h[N] > 0. */
static double lambda_loglik(const double* h, int n_max, double lambda0, double lam) {
  double mx = -INFINITY;
  for (int k = 0; k <= n_max; ++k) {
    if (!(h[k] > 0.0)) continue;
    double t = (k == 0) ? log(h[k]) : (lam > 0.0 ? log(h[k]) + k * log(lam / lambda0) : -INFINITY);
    if (t > mx) mx = t;
  }
  if (mx == -INFINITY) return -INFINITY;
  double acc = 0.0;
  for (int k = 0; k <= n_max; ++k) {
    if (!(h[k] > 0.0)) continue;
    double t = (k == 0) ? log(h[k]) : (lam > 0.0 ? log(h[k]) + k * log(lam / lambda0) : -INFINITY);
    acc += exp(t - mx);
  }
  return -lam + mx + log(acc);
}

/* l'(lambda) = -1 + (sum_N N w_N) / (lambda sum_N w_N), w_N = h[N] (lambda / lambda0)^N */
static double lambda_dloglik(const double* h, int n_max, double lambda0, double lam) {
  double mx = -INFINITY;
  for (int k = 0; k <= n_max; ++k)
    if (h[k] > 0.0) {
      double t = log(h[k]) + k * log(lam / lambda0);
      if (t > mx) mx = t;
    }
  double sw = 0.0, snw = 0.0;
  for (int k = 0; k <= n_max; ++k)
    if (h[k] > 0.0) {
      double e = exp(log(h[k]) + k * log(lam / lambda0) - mx);
      sw += e;
      snw += k * e;
    }
  return -1.0 + snw / (lam * sw);
}

/* ------------------------------------------------------------------------------------
 * The Wasserstein distance the convergence check of Sec. 3.2 uses on PE sequences.
 * ---------------------------------------------------------------------------------- */
static int cmp_double(const void* x, const void* y) {
  const double a = *(const double*)x, b = *(const double*)y;
  return (a > b) - (a < b);
}

double orc_wasserstein1(const double* a, int na, const double* b, int nb) {
  /* W1 on the line is the area between the two CDFs: walk the merged sorted points, and on
   * each interval between consecutive points add |F_a - F_b| times its length */
  double* sa = (double*)malloc(sizeof(double) * (size_t)na);
  double* sb = (double*)malloc(sizeof(double) * (size_t)nb);
  if (!sa || !sb) { free(sa); free(sb); return NAN; }
  memcpy(sa, a, sizeof(double) * (size_t)na);
  memcpy(sb, b, sizeof(double) * (size_t)nb);
  qsort(sa, (size_t)na, sizeof(double), cmp_double);
  qsort(sb, (size_t)nb, sizeof(double), cmp_double);
  int i = 0, j = 0;
  double x = fmin(sa[0], sb[0]), area = 0.0;
  while (i < na || j < nb) {
    /* the next point of either sample; both CDFs are constant on [x, next) */
    const double next = (j >= nb || (i < na && sa[i] <= sb[j])) ? sa[i] : sb[j];
    area += fabs((double)i / na - (double)j / nb) * (next - x);
    x = next;
    while (i < na && sa[i] == x) ++i;
    while (j < nb && sb[j] == x) ++j;
  }
  free(sa);
  free(sb);
  return area;
}

double orc_pe_wasserstein(const double* v, int N) {
  /* the sequence with its dummy PE at 0 against the dummy alone */
  double* a = (double*)malloc(sizeof(double) * ((size_t)N + 1));
  if (!a) return NAN;
  a[0] = 0.0;
  for (int k = 0; k < N; ++k) a[k + 1] = v[k];
  const double zero = 0.0;
  const double d = orc_wasserstein1(a, N + 1, &zero, 1);
  free(a);
  return d;
}

double orc_lambda_mle(const double* h, int n_max, double lambda0) {
  int top = -1;
  for (int k = 0; k <= n_max; ++k)
    if (h[k] > 0.0) top = k;
  if (top < 0) return NAN;
  if (top == 0) return 0.0;
  const double hi = 2.0 * top + 10.0;
  const int G = 20000;
  int best = 0;
  double bl = -INFINITY;
  for (int g = 0; g <= G; ++g) {
    double l = lambda_loglik(h, n_max, lambda0, hi * g / G);
    if (l > bl) { bl = l; best = g; }
  }
  /* bisection on l'(lambda) = -1 + E_w[N] / lambda, w_N = h[N] (lambda / lambda0)^N, inside the
   * bracket around the best grid point (l' changes sign at the maximum) */
  double a = hi * (best > 0 ? best - 1 : 0) / G, b = hi * (best < G ? best + 1 : G) / G;
  if (a <= 0.0) a = 1e-300;
  for (int it = 0; it < 400 && b - a > 4e-16 * b; ++it) {
    const double m = 0.5 * (a + b);
    if (lambda_dloglik(h, n_max, lambda0, m) > 0.0) a = m; else b = m;
  }
  double x = 0.5 * (a + b);
  /* the maximum may sit on the boundary lambda = 0 */
  if (lambda_loglik(h, n_max, lambda0, 0.0) >= lambda_loglik(h, n_max, lambda0, x)) return 0.0;
  return x;
}

int orc_run_batch(const orc_params* p, const orc_batch* b, int mode, int n_threads,
                  orc_summary* out, orc_trace* trace) {
  model M;
  double* V = NULL;
  int rc = build_model(p, &M, &V);
  if (rc) return rc;
  if (b->n_steps < 0 || b->burn_in < 0 || b->n_waveforms < 0) { free(V); return ORC_ERR_INVALID; }
  if (n_threads < 1) n_threads = 1;
  if (n_threads > b->n_waveforms) n_threads = b->n_waveforms > 0 ? b->n_waveforms : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  worker_arg* args = (worker_arg*)malloc(sizeof(worker_arg) * n_threads);
  if (!th || !args) { free(th); free(args); free(V); return ORC_ERR_NOMEM; }
  for (int t = 0; t < n_threads; ++t) {
    args[t].p = p; args[t].M = &M; args[t].b = b; args[t].mode = mode;
    args[t].tid = t; args[t].nthreads = n_threads; args[t].out = out; args[t].trace = trace;
    args[t].rc = 0;
  }
  if (n_threads == 1) {
    worker(&args[0]);
  } else {
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &args[t]);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  }
  for (int t = 0; t < n_threads; ++t) if (args[t].rc) rc = args[t].rc;
  free(th); free(args); free(V);
  return rc;
}

int orc_run_chain_state(const orc_params* p, const orc_batch* b, int mode,
                        orc_summary* out, orc_trace* trace, int32_t* list_out, int32_t* N_out,
                        int32_t* k0_out, double* sinv_out, double* y_out, double* logdet_out,
                        int32_t* e_out) {
  model M;
  double* V = NULL;
  int rc = build_model(p, &M, &V);
  if (rc) return rc;
  chain_in c;
  rc = make_chain_in(p, &M, b, 0, mode, &c);
  if (rc == 0) rc = run_chain(&c, out, trace, list_out, N_out, k0_out, sinv_out, y_out, logdet_out, e_out);
  free(V);
  return rc;
}

double orc_logp_definition_e(const orc_params* p, const float* w, int n, const int32_t* j, const int32_t* e,
                             int N, double* logdet_out, double* quad_out) {
  model M;
  double* V = NULL;
  if (build_model(p, &M, &V) != 0) return NAN;
  double r = logp_def(&M, w, n, j, e, N, logdet_out, quad_out, NULL);
  free(V);
  return r;
}

double orc_logp_definition(const orc_params* p, const float* w, int n, const int32_t* j, int N,
                           double* logdet_out, double* quad_out) {
  return orc_logp_definition_e(p, w, n, j, NULL, N, logdet_out, quad_out);
}

int orc_delta_nu_e(const orc_params* p, const float* w, int n, const int32_t* j, const int32_t* e, int N,
                   int kind, int k, int jp, int ep, int mode, double* dnu_out) {
  model M;
  double* V = NULL;
  int rc = build_model(p, &M, &V);
  if (rc) return rc;
  if ((kind != 0 && (k < 0 || k >= N)) || N < 0) { free(V); return ORC_ERR_INVALID; }
  int32_t* e0 = (int32_t*)calloc((size_t)N + 1, sizeof(int32_t));
  if (!e0) { free(V); return ORC_ERR_NOMEM; }
  if (e) memcpy(e0, e, sizeof(int32_t) * N);
  if (mode == ORC_MODE_DEFINITION) {
    int32_t* z2 = (int32_t*)malloc(sizeof(int32_t) * (N + 1));
    int32_t* e2 = (int32_t*)malloc(sizeof(int32_t) * (N + 1));
    memcpy(z2, j, sizeof(int32_t) * N);
    memcpy(e2, e0, sizeof(int32_t) * N);
    int N2 = N;
    if (kind == 0) { z2[N] = jp; e2[N] = ep; N2 = N + 1; }
    else if (kind == 1) { z2[k] = j[N - 1]; e2[k] = e0[N - 1]; N2 = N - 1; }
    else { z2[k] = jp; e2[k] = ep; }
    double l0 = logp_def(&M, w, n, j, e0, N, NULL, NULL, NULL);
    double l1 = logp_def(&M, w, n, z2, e2, N2, NULL, NULL, NULL);
    free(z2);
    free(e2);
    *dnu_out = l1 - l0;
  } else {
    inc_state st;
    memset(&st, 0, sizeof(st));
    if (inc_init(&st, p, w, n) != 0) { inc_free(&st); free(e0); free(V); return ORC_ERR_NOMEM; }
    double d;
    /* Sigma^-1(z) built from the empty state by successive births (Eq. (12), a_- = 0) */
    for (int i = 0; i < N; ++i) {
      for (int x = 0; x < n; ++x) st.am[x] = 0.0;
      pe_vector(&M, n, j[i], st.ap);
      if (inc_delta_nu(&st, p, e0[i], e0[i], &d) != 0) { inc_free(&st); free(e0); free(V); return ORC_ERR_INVALID; }
      inc_accept(&st, p);
    }
    int em = ep, epp = ep;
    if (kind == 0) { for (int x = 0; x < n; ++x) st.am[x] = 0.0; pe_vector(&M, n, jp, st.ap); }
    else if (kind == 1) { pe_vector(&M, n, j[k], st.am); for (int x = 0; x < n; ++x) st.ap[x] = 0.0; em = epp = e0[k]; }
    else { pe_vector(&M, n, j[k], st.am); pe_vector(&M, n, jp, st.ap); em = e0[k]; }
    rc = inc_delta_nu(&st, p, em, epp, &d);
    inc_free(&st);
    if (rc) { free(e0); free(V); return ORC_ERR_INVALID; }
    *dnu_out = d;
  }
  free(e0);
  free(V);
  return 0;
}

int orc_delta_nu(const orc_params* p, const float* w, int n, const int32_t* j, int N,
                 int kind, int k, int jp, int mode, double* dnu_out) {
  return orc_delta_nu_e(p, w, n, j, NULL, N, kind, k, jp, 0, mode, dnu_out);
}

int orc_lucyddm(const orc_params* p, const float* w, int n, double t_origin, int n_iter, double thresh,
                double* q_out, int32_t* z_out, int z_cap, int32_t* n_z, int32_t* T_lo, int32_t* T_hi,
                double* t0_out) {
  if (!w || n < 1 || n_iter < 0 || z_cap < 0 || (z_cap > 0 && !z_out) || !n_z || !T_lo || !T_hi || !t0_out)
    return ORC_ERR_INVALID;
  model M;
  double* V = NULL;
  int rc = build_model(p, &M, &V);
  if (rc) return rc;
  rc = lucyddm(&M, w, n, t_origin, n_iter, thresh, q_out, z_out, z_cap, n_z, T_lo, T_hi, t0_out);
  free(V);
  return rc;
}
